/*
 * spca.h -- C ABI of the GB300 (sm_103a) alternating-maximization sparse PCA library
 * (libspca.so).
 *
 * The library computes, for one data matrix A (n samples x p variables; dense, or sparse
 * in compressed sparse rows), the single-component sparse PCA problem
 * OPT = max_{x in X} f(x) for any of the eight formulations of Table 1 of Richtarik,
 * Jahani, Ahipasaoglu, Takac, "Alternating maximization: unifying framework for 8 sparse
 * PCA formulations and efficient parallel codes" (arXiv 1212.4137), by the alternating
 * maximization method of Algorithm 2 run from r starting points at once (Section 4: the r
 * matrix-vector products of a sweep become matrix-matrix products), keeping the best start.
 *
 * Conventions (all entry points):
 *   - every call returns an int status (spca_status); no exception crosses the ABI;
 *   - outputs are left untouched when a call fails;
 *   - "host" buffers are ordinary (pageable or pinned) host memory, "device" buffers are
 *     CUDA device memory of the handle's device;
 *   - matrices are row-major; a block of r vectors of length m is r x m row-major (one
 *     vector per row);
 *   - a handle is bound to one CUDA stream and is not thread-safe.  Work is queued on
 *     that stream; spca_solve returns after its results are on the host.
 * There is no CPU fallback: without a usable GB300 the calls fail with SPCA_E_CUDA.
 */
#ifndef SPCA_H
#define SPCA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spca_handle spca_handle;

/* status codes */
typedef enum {
    SPCA_OK = 0,
    SPCA_E_INVALID = 1,      /* an argument is out of range, a pointer is NULL, A is not finite */
    SPCA_E_NOMEM = 2,        /* a device or pinned-host allocation failed                         */
    SPCA_E_CUDA = 3,         /* a CUDA runtime error (no device, launch failure, ...)             */
    SPCA_E_TIMEOUT = 4,      /* a bounded device-side wait gave up (reported by the kernel)       */
    SPCA_E_BUSY = 5,         /* the handle is in use                                              */
    SPCA_E_UNSUPPORTED = 6   /* a valid request the library does not implement                     */
} spca_status;

/* element types (the low-precision storage is FP16 with power-of-two row scales rather than
 * BF16: the same bytes and tensor-core rate, three more significant bits, and the row scales
 * cover the range BF16's wider exponent would) */
typedef enum {
    SPCA_F32 = 0,
    SPCA_F64 = 1,
    SPCA_FP16 = 2,            /* storage only: a 16-bit FP16 copy of A, row-scaled (see spca_create) */
    SPCA_FP8_E4M3_COLSCALED = 3,
    SPCA_FP16_RESIDENT = 4    /* storage only: A held only in 16 bits (see spca_create)             */
} spca_dtype;

/* formulation numbers = Table 1 of the paper:
 *   #  variance  sparsity   usage        X                                  f(x)
 *   1  L2        L0         constraint   ||x||_2 <= 1, ||x||_0 <= s         ||Ax||_2
 *   2  L1        L0         constraint   ||x||_2 <= 1, ||x||_0 <= s         ||Ax||_1
 *   3  L2        L1         constraint   ||x||_2 <= 1, ||x||_1 <= sqrt(s)   ||Ax||_2
 *   4  L1        L1         constraint   ||x||_2 <= 1, ||x||_1 <= sqrt(s)   ||Ax||_1
 *   5  L2        L0         penalty      ||x||_2 <= 1                       ||Ax||_2^2 - gamma ||x||_0
 *   6  L1        L0         penalty      ||x||_2 <= 1                       ||Ax||_1^2 - gamma ||x||_0
 *   7  L2        L1         penalty      ||x||_2 <= 1                       ||Ax||_2   - gamma ||x||_1
 *   8  L1        L1         penalty      ||x||_2 <= 1                       ||Ax||_1   - gamma ||x||_1 */
typedef enum {
    SPCA_L2_L0CON = 1, SPCA_L1_L0CON = 2, SPCA_L2_L1CON = 3, SPCA_L1_L1CON = 4,
    SPCA_L2_L0PEN = 5, SPCA_L1_L0PEN = 6, SPCA_L2_L1PEN = 7, SPCA_L1_L1PEN = 8
} spca_formulation;

/* gamma modes of the penalty forms 5..8.
 *   SPCA_GAMMA_FIXED       gamma as given (Algorithm 2).
 *   SPCA_GAMMA_TARGET_NNZ  the sparsity-targeting rule of Section 4.1: during the first
 *                          gamma_calib_sweeps sweeps each start sets gamma so that exactly
 *                          s entries survive (the (s+1)-th largest v_i^2 for U_gamma, the
 *                          (s+1)-th largest |v_i| for V_gamma; 0 if s >= p), then freezes it. */
typedef enum { SPCA_GAMMA_FIXED = 0, SPCA_GAMMA_TARGET_NNZ = 1 } spca_gamma_mode;

/* per-start termination status */
typedef enum {
    SPCA_ST_MAXITER = 0,     /* ran max_iter sweeps                                           */
    SPCA_ST_CONVERGED = 1,   /* stopping rule of Section 2.2 met: F_{k+1} <= (1 + tol) F_k     */
    SPCA_ST_DEGENERATE = 2   /* the x-step returned 0 (or Ax = 0 for L2 variance): x = 0       */
} spca_start_status;

/* compute engines for the two contractions of a sweep */
typedef enum {
    SPCA_ENGINE_AUTO = 0,    /* tensor cores for low-precision sweeps, and for n p r >= 2^26  */
                             /* unless the starts are few (r <= 8: the CUDA cores' streaming  */
                             /* GEMV reads A once per product at HBM speed); else CUDA cores  */
                             /* (their per-sweep fixed costs dominate small work)             */
    SPCA_ENGINE_SIMT = 1,    /* FP32 CUDA-core kernels                                        */
    SPCA_ENGINE_TC = 2,      /* tcgen05 tensor-core kernels (TMEM accumulators, TMA loads)    */
    SPCA_ENGINE_TC_LOWP = 3  /* spca_products only: the tensor cores on the low-precision      */
                             /* copies (as in the first lowp_sweeps sweeps of a solve)         */
} spca_engine;

/*
 * spca_create -- copy A to the device and prepare the layouts the kernels read.
 *   out          receives the new handle (host pointer to a handle pointer).
 *   A            n x p row-major matrix with leading dimension lda >= p (elements), of type
 *                in_dtype (SPCA_F32 or SPCA_F64), in host memory (a_is_device = 0) or
 *                device memory (a_is_device = 1).  Copied; the caller may free it on return.
 *                The library does not centre the columns (the paper assumes centred data,
 *                Section 1).
 *   storage      SPCA_F32, SPCA_FP16 (a 16-bit copy for the low-precision sweeps,
 *                spca_params.lowp_sweeps) or SPCA_FP8_E4M3_COLSCALED.  All keep the FP32 master
 *                copy and the tensor-core operand format: two FP16 planes of a row-scaled copy
 *                (hi + lo carries 22 significant bits); the 16-bit copy is the leading plane
 *                (A rounded to 11 significant bits with one power-of-two scale per row), which
 *                the low-precision sweeps of SPCA_F32 and SPCA_FP16 handles read.
 *                SPCA_FP8_E4M3_COLSCALED adds E4M3 copies of A and of A^T with power-of-two
 *                scales per row of A and per column of A (A rounded to 4 significant bits; the
 *                largest entry of a row or column in [128, 256)); the low-precision sweeps then
 *                run the tensor cores' 8-bit kind (y in E4M3 at scale 2^7, x per row scaled)
 *                and an 8-bit support gather, accumulating in FP32 (a clone's low-precision
 *                sweeps read the FP16 leading plane instead).  Both 16- and 8-bit storage need
 *                tensor cores (sm_100+): SPCA_E_UNSUPPORTED otherwise.
 *                SPCA_FP16_RESIDENT keeps nothing but the leading FP16 planes of A and of A^T
 *                with their row scales: 4 bytes per entry of A on the device instead of 16 (the
 *                FP32 copies and the second planes are freed once the planes are built).  The
 *                matrix the solves see is that 16-bit copy: every sweep is a low-precision sweep
 *                (one tensor-core product per tile on the leading planes of A and of x or y, the
 *                FP16 support gather), the stopping rule applies from the second sweep on, and
 *                the objective of the finalise is that of the copy of A^T (FP16 entries times
 *                their column's power-of-two scale), accumulated as for SPCA_F32.  Such a handle
 *                takes the tensor-core engine only and no low-precision options (spca_solve),
 *                on-the-fly replacement or deflation, and spca_products only with
 *                SPCA_ENGINE_TC_LOWP (SPCA_E_UNSUPPORTED / SPCA_E_INVALID otherwise).
 *   cuda_stream  the caller's cudaStream_t (NULL = the legacy default stream): every call on
 *                the handle starts after the work queued on it before the call and returns with
 *                its own work complete.  The handle runs its kernels on a stream of its own, so
 *                that the sweeps of a solve can be captured into CUDA graphs and replayed.
 * Errors: SPCA_E_INVALID (NULL pointers, n < 1, p < 1, lda < p, A not finite, unknown dtype),
 *         SPCA_E_UNSUPPORTED (n above 16,776,960 = 65535 * 256 rows: the finalise takes a dense
 *         A's rows in blocks of 256 on a grid dimension of at most 65535; SPCA_F64 storage;
 *         16- or 8-bit storage without tensor cores), SPCA_E_NOMEM, SPCA_E_CUDA.
 */
int spca_create(spca_handle **out, const void *A, int64_t n, int64_t p, int64_t lda,
                int in_dtype, int a_is_device, int storage, void *cuda_stream);

/*
 * spca_create_csr -- the same for a sparse A given in compressed sparse rows, the layout of the
 * text corpora of Section 5 (document x word counts).  The handle keeps A by rows and by
 * columns, each canonical (indices ascending within a row, repeated entries summed), in FP32;
 * no dense copy is made.  The sweeps run on sparse CUDA-core kernels: u = A x over the stored
 * entries (by rows) for a dense x, or over the columns of x's support (by columns) once x is
 * sparse; v = A^T y over the stored entries (by columns); the finalise by rows in compensated
 * FP32 pairs.
 *   n, p         rows and columns, 1 .. 2^31 - 1.
 *   nnz          stored entries, 0 .. 2^31 - 1 (= row_ptr[n]).
 *   row_ptr      n + 1 int64 offsets: row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz.
 *   col_idx      nnz int32 column indices in [0, p), in any order within a row; a repeated
 *                (row, column) pair adds up.
 *   values       nnz finite floats.
 *   is_device    the three arrays are in device memory (1) or host memory (0).  Either way they
 *                are copied (device input through the host, where the layouts are built) and
 *                may be freed on return.
 *   cuda_stream  as in spca_create.
 * On such a handle spca_solve and spca_products take SPCA_ENGINE_AUTO or SPCA_ENGINE_SIMT
 * (SPCA_ENGINE_TC and lowp_sweeps > 0 are SPCA_E_UNSUPPORTED); spca_deflate keeps A sparse and
 * holds the deflations as a low-rank update (see spca_deflate).
 * Errors: SPCA_E_INVALID (NULL pointers, sizes out of range, row_ptr malformed, a column out of
 *         range, a value or a sum of repeated values not finite), SPCA_E_NOMEM, SPCA_E_CUDA.
 */
int spca_create_csr(spca_handle **out, int64_t n, int64_t p, int64_t nnz, const int64_t *row_ptr,
                    const int32_t *col_idx, const float *values, int is_device, void *cuda_stream);

/*
 * spca_clone -- a new handle on the matrix another handle holds, for solves on several streams or
 * host threads at once (one handle per thread: a handle is not thread-safe).  The clone shares
 * the source's device copies of A and their layouts, read-only, and has its own stream, workspace
 * and captured graphs; the matrix is freed with the last handle that holds it.  While a matrix
 * is shared, spca_deflate on any of its handles is SPCA_E_UNSUPPORTED.  A clone's contractions
 * run on the cluster kernel: the pair kernel's stream-K schedule needs every CTA of a launch
 * resident at once, which launches of other handles at the same time cannot guarantee (the
 * source handle keeps stream-K; solve on clones alone while several run together).
 *   out          receives the new handle.
 *   src          a handle from spca_create, spca_create_csr or spca_clone.
 *   cuda_stream  as in spca_create.
 * Errors: SPCA_E_INVALID, SPCA_E_NOMEM, SPCA_E_CUDA.
 */
int spca_clone(spca_handle **out, spca_handle *src, void *cuda_stream);

/*
 * Parameters of one solve (Algorithm 2 from r starts, Section 2.2 stopping rule).
 *   form                Table 1 formulation (1..8).
 *   s                   L0 forms 1, 2: the cardinality bound (integer 1..p).
 *                       L1 forms 3, 4: the L1 radius is sqrt(s), s >= 1.
 *                       penalty forms in SPCA_GAMMA_TARGET_NNZ mode: the target count (1..p).
 *   gamma               penalty forms, SPCA_GAMMA_FIXED mode: gamma >= 0.
 *   gamma_mode          spca_gamma_mode (penalty forms only).
 *   gamma_calib_sweeps  sweeps during which gamma is re-targeted (>= 1; typical 10).
 *   r                   number of starts (1 .. 65535; several kernels put the starts on a
 *                       grid dimension of at most 65535: SPCA_E_UNSUPPORTED above).
 *   max_iter            maximum sweeps per start (>= 1).
 *   tol                 stopping tolerance; a start stops after sweep k >= 2 when
 *                       F(x^(k), y^(k-1)) <= (1 + tol) F(x^(k-1), y^(k-2)), comparing only
 *                       values computed with the same gamma; tol < 0 disables the test.
 *   seed                starts when x0 == NULL: x^(0) = g / ||g||_2 with g the Box-Muller
 *                       normals of the counter-based SplitMix64 stream (seed, stream 5);
 *                       element (c, j) of the r x p block is normal number c*p + j.
 *   x0_is_device        x0 is a device pointer (1) or a host pointer (0).
 *   engine              spca_engine.
 *   lowp_sweeps         lowp_sweeps sweeps (after the first lowp_first ones) read A rounded to
 *                       11 significant bits
 *                       (the leading FP16 plane: one tensor-core product per tile in v = A^T y
 *                       and u = A x, and an FP16 support gather), y's leading plane, FP32
 *                       accumulation;
 *                       no start stops during them.  Then FP32 sweeps refine every start
 *                       to the stopping rule.  0 = FP32 throughout.  Needs the tensor-core
 *                       engine (SPCA_E_UNSUPPORTED otherwise).
 *   lowp_first          FP32 sweeps before the low-precision ones (0 = the low-precision
 *                       sweeps come first).  The early sweeps decide which stationary point a
 *                       start reaches; running them in FP32 keeps each start on its FP32 path.
 *   refine_sweeps       at most this many FP32 sweeps after the low-precision ones
 *                       (0 = up to max_iter sweeps in all).
 *   timeout_us          wall-clock limit of the solve in microseconds (0 = none), checked
 *                       each time the host reads the active count back (every 4 sweeps):
 *                       past it the solve returns SPCA_E_TIMEOUT and writes no result.
 *   total_starts        on-the-fly replacement (Section 4.3): with total_starts > r the solve
 *                       runs total_starts starts through r slots, a slot taking the next start
 *                       (in index order) in the sweep its start stops; x0 then holds
 *                       total_starts rows (the seeded start c is normal numbers c*p + j), the
 *                       start_* outputs hold total_starts entries, and max_iter bounds each
 *                       start's sweeps.  0 (or <= r) = all r starts at once.  At most 65535
 *                       (SPCA_E_UNSUPPORTED above).  Not combined with lowp_sweeps
 *                       (SPCA_E_UNSUPPORTED).
 */
typedef struct {
    int form;
    double s;
    double gamma;
    int gamma_mode;
    int gamma_calib_sweeps;
    int r;
    int max_iter;
    double tol;
    uint64_t seed;
    int x0_is_device;
    int engine;
    int lowp_sweeps;
    int refine_sweeps;
    int64_t timeout_us;
    int total_starts;
    int lowp_first;
} spca_params;

/*
 * Results of one solve.  Scalars are always written.  Every pointer is a caller-owned
 * HOST buffer of the stated length, or NULL to skip that output.
 *   objective            f(x) of Table 1 for the best start, accumulated in FP64 on the GPU
 *                        (gamma = the start's final gamma for the penalty forms).
 *   explained_variance   ||Ax||_2^2 (L2 variance) or ||Ax||_1 (L1 variance) of the best start.
 *   best_start           argmax over starts of the objective (of the explained variance in
 *                        SPCA_GAMMA_TARGET_NNZ mode, where gammas differ per start); ties go
 *                        to the lower start index.
 *   sweeps_total         sum over starts of sweeps performed (sweeps x starts of work).
 *   x [p], y [n]         the best start's normalised x and y = y(x) (S1 or S2 of Table 3).
 *   support [p]          indices of the nonzeros of x, ascending; nnz entries are written.
 *   start_* [r]          per-start objective, explained variance, last F value, sweeps,
 *                        status (spca_start_status), final gamma ([total_starts] with
 *                        on-the-fly replacement).
 *   start_x [r*p]        every start's final x, one per row ([total_starts*p] likewise).
 */
typedef struct {
    double objective;
    double explained_variance;
    double gamma;
    int best_start;
    int best_iters;
    int best_status;
    int converged;
    int degenerate;
    int64_t sweeps_total;
    int64_t nnz;
    float *x;
    float *y;
    int64_t *support;
    double *start_objective;
    double *start_explained;
    double *start_F;
    int *start_iters;
    int *start_status;
    double *start_gamma;
    float *start_x;
} spca_result;

/*
 * spca_solve -- Algorithm 2 (Section 2.2) for r starts at once, then the Table 1 objective
 * of every start in FP64 and the best start.
 *   x0   r x p starting vectors (one per row, need not be normalised) of type float, host or
 *        device memory per prm->x0_is_device; NULL = seeded starts (see spca_params.seed).
 * Errors: SPCA_E_INVALID (NULL h/prm/res, form outside 1..8, s outside [1, p] for L0 or
 *         target modes, s < 1 for L1 constraints, gamma < 0, r < 1, max_iter < 1,
 *         gamma_calib_sweeps < 1 in target mode, unknown engine, non-finite x0),
 *         SPCA_E_UNSUPPORTED (engine not available), SPCA_E_NOMEM, SPCA_E_CUDA,
 *         SPCA_E_TIMEOUT.
 */
int spca_solve(spca_handle *h, const spca_params *prm, const float *x0, spca_result *res);

/*
 * spca_xstep -- the x-step of Algorithm 2 (Table 3, S3..S6, then normalisation) on r
 * given vectors v = A^T y, on the handle's stream, device memory only.  Exposed so that
 * each operator (T_s, U_gamma, V_gamma, lambda_s) can be checked on its own.
 *   form, s, gamma   as in spca_params; calibrate != 0 applies the Section 4.1 rule
 *                    (penalty forms) before thresholding.
 *   V     device, r x p float, leading dimension ldv >= p.
 *   X     device, r x p float output (ldx >= p): the normalised x-step result, or 0.
 *   F     device, r doubles: the Table 3 value of the subproblem.
 *   nnz   device, r ints: nonzeros of each result.
 *   thr   device, r doubles: the threshold used (gamma for U/V, lambda_s for S4, 0 for T_s).
 * Errors: SPCA_E_INVALID, SPCA_E_CUDA.
 */
int spca_xstep(spca_handle *h, int form, double s, double gamma, int calibrate,
               const float *V, int64_t ldv, int r, float *X, int64_t ldx,
               double *F, int *nnz, double *thr);

/*
 * spca_products -- the linear algebra of one sweep of Algorithm 2 for r given iterates, on
 * the handle's stream, device memory only: u = A x (dense contraction), the y-step (S1 for
 * L2 variance, S2 with sgn(0) = +1 for L1 variance, chosen by `form`), and v = A^T y.
 * Exposed so that the contractions of each engine can be checked on their own.
 *   form    Table 1 formulation (only its variance norm matters here).
 *   engine  spca_engine; SPCA_ENGINE_TC_LOWP runs both contractions as a low-precision sweep
 *           does (the leading FP16 planes, or the E4M3 copies of an FP8 handle), to check them.
 *   X       device, r x p float iterates (ldx >= p).
 *   U       device, r x n float output u = A x (ldu >= n).
 *   V       device, r x p float output v = A^T y (ldv >= p); unspecified for a row whose
 *           u is 0 under L2 variance.
 * Errors: SPCA_E_INVALID, SPCA_E_UNSUPPORTED (engine; r above 65535), SPCA_E_NOMEM, SPCA_E_CUDA,
 *         SPCA_E_TIMEOUT.
 */
int spca_products(spca_handle *h, int form, int engine, const float *X, int64_t ldx, int r,
                  float *U, int64_t ldu, float *V, int64_t ldv);

/*
 * spca_deflate -- projection deflation of the handle's matrix for a further component:
 * A <- A (I - z z^T) with z = x / ||x||_2 (the paper computes several components, Section 1,
 * without fixing a deflation scheme).  The next spca_solve on the handle then works on the
 * deflated matrix, so z is not found again.  Dense A: w = A z is accumulated as compensated FP32
 * pairs, each entry updated in FP64 and rounded once to FP32; the transposed copy and the
 * tensor-core operands are rebuilt.  Sparse A (spca_create_csr): A stays as given and the
 * deflations are kept as A_k = A - W Z^T (z_i in FP32, w_i = A_{i-1} z_i in compensated FP32
 * pairs, rounded once); every sweep subtracts W (Z^T x) from u and Z (W^T y) from v, and the
 * finalise subtracts W (Z^T x) in pair arithmetic.  Synchronous on the handle's stream.
 *   x            p floats (typically spca_result.x of the last solve), host memory
 *                (x_is_device = 0) or device memory (x_is_device = 1); need not be normalised.
 * Errors: SPCA_E_INVALID (NULL pointers, x not finite or zero: A is then unchanged),
 *         SPCA_E_NOMEM, SPCA_E_CUDA.
 */
int spca_deflate(spca_handle *h, const float *x, int x_is_device);

/*
 * Measurement hooks (not part of the method): per-kernel launch counts are always kept;
 * with profiling on, the launches of the selected kernel ids are also bracketed by CUDA
 * events on the handle's stream (each pair costs a few microseconds of host and device time).
 *   spca_profile_enable  mask = bit (1 << id) per spca_kernel_id to time, SPCA_PROFILE_ALL for
 *                        every kernel, 0 to stop; clears the counters.  A mask outside
 *                        0..SPCA_PROFILE_ALL is SPCA_E_INVALID.
 *   spca_profile_query   kernel = one of spca_kernel_id, or SPCA_K_ALL for the total launch
 *                        count (ms then = sum over kernels); waits for the stream, then
 *                        writes the number of launches and their summed device time in ms
 *                        (0 while profiling is off).  Either output pointer may be NULL.
 * Errors: SPCA_E_INVALID (NULL handle, unknown kernel id), SPCA_E_CUDA.
 */
typedef enum {
    SPCA_K_ALL = -1,
    SPCA_K_INIT = 0,          /* a1: start normalisation                                   */
    SPCA_K_U_DENSE = 1,       /* a2: u = A x, dense contraction                            */
    SPCA_K_U_SPARSE = 2,      /* a2: u = A x over the support of x                          */
    SPCA_K_YSTEP = 3,         /* a3: y-step (S1 / S2)                                       */
    SPCA_K_V = 4,             /* a4: v = A^T y                                              */
    SPCA_K_XSTEP = 5,         /* a5, a6: x-step, F, stopping rule                           */
    SPCA_K_FINALISE = 6,      /* a7: FP64 objective, best start, outputs                    */
    SPCA_K_PREP = 7,          /* layout preparation and input checks                        */
    SPCA_K_COUNT = 8
} spca_kernel_id;
#define SPCA_PROFILE_ALL ((1 << SPCA_K_COUNT) - 1)
int spca_profile_enable(spca_handle *h, int mask);
int spca_profile_query(spca_handle *h, int kernel, int64_t *launches, double *ms);

/*
 * spca_objective_noalloc -- the objective and the explained variance of r given vectors x,
 * with u = A x accumulated in FP64: the values spca_solve reports per start (start_objective,
 * start_explained).  Per formulation the objective is
 *   1, 3: ||Ax||_2          2, 4: ||Ax||_1
 *   5:    ||Ax||_2^2 - gamma ||x||_0      6: ||Ax||_1^2 - gamma ||x||_0
 *   7:    ||Ax||_2 - gamma ||x||_1        8: ||Ax||_1 - gamma ||x||_1
 * and the explained variance ||Ax||_2^2 (odd forms) or ||Ax||_1 (even forms).  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate device memory -- code
 * running inside someone else's CUDA graph capture (an allocation there is an error or breaks
 * the capture), under an allocator or memory pool that owns the whole device, or in a
 * latency-critical loop where an allocation's implicit synchronisation is not acceptable.  It
 * needs no handle and allocates nothing: its scratch is a fixed array in the library's device
 * memory (4 MiB, held on every GPU that loads the library until the process exits).
 *   form, gamma  formulation (1..8) and the penalty weight (>= 0; ignored by 1..4).
 *   A            device, n x p float, row-major, leading dimension lda >= p.
 *   X            device, r x p float, one vector per row, leading dimension ldx >= p.
 *   f, ev        device, r doubles each (outputs).
 *   cuda_stream  cudaStream_t the kernels are queued on (NULL = the legacy default stream);
 *                the call returns once they are queued.
 * Limits: r * ceil(n / 256) <= SPCA_NOALLOC_MAX_PARTIALS (the scratch), else SPCA_E_INVALID
 * and nothing runs; r <= 65535 (a grid dimension), else SPCA_E_UNSUPPORTED.
 * The first call on a device looks up the scratch's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  Every call shares the
 * one scratch array: calls whose kernels overlap on the GPU (other streams, other threads)
 * race and must be serialised by the caller.  The scratch keeps the last call's contents; each
 * call writes every entry it reads.
 * Errors: SPCA_E_INVALID (form, sizes, leading dimensions, NULL pointers, gamma, scratch limit),
 *         SPCA_E_UNSUPPORTED (r above 65535), SPCA_E_CUDA.
 */
#define SPCA_NOALLOC_MAX_PARTIALS 262144
int spca_objective_noalloc(int form, double gamma, const float *A, int64_t n, int64_t p, int64_t lda,
                           const float *X, int64_t ldx, int r, double *f, double *ev,
                           void *cuda_stream);

/*
 * spca_set_waits -- the bounded device-side waits of the handle's tensor-core contractions.
 * Every wait inside those kernels (a pipeline stage, the accumulator, the part of a split tile
 * that another CTA pair computes) gives up after wait_limit_us microseconds: the kernel records
 * SPCA_E_TIMEOUT, lets the loads it has in flight land, frees its tensor memory and returns, and
 * the call that launched it returns SPCA_E_TIMEOUT; the handle stays usable.  This is the
 * failure detection of the device side: a stalled CTA pair turns into an error status instead
 * of a kernel that never ends.  Not part of the method (the paper has no counterpart).
 *   wait_limit_us      1 .. 60,000,000 (the default is 2,000,000: 2 s).
 *   unpublished_parts  test switch: nonzero makes the CTAs that finish a split tile wait for a
 *                      part flag that no CTA ever sets, so that their waits run out and the
 *                      timeout path above runs; 0 for normal work.
 * Captured sweep graphs are dropped (they hold the old settings).
 * Errors: SPCA_E_INVALID (NULL handle, limit out of range).
 */
int spca_set_waits(spca_handle *h, int64_t wait_limit_us, int unpublished_parts);

/*
 * Groups of problems: Algorithm 2 for many independent problems at once, each with its own
 * matrix (a handle), formulation, s or gamma and starts (the batching of Section 4 carried across
 * problems).  Every phase of a sweep is one launch over all the group's problems: the dense
 * u = A x of a problem's first sweep and v = A^T y of every sweep as one persistent tensor-core
 * launch over the tiles of all problems; the start set-up, support gather, y-step, x-step (the
 * candidate filter and operator, then the full pass for the starts they leave) and active lists
 * as one launch each over all starts or problems.  Each problem's results do not depend on the
 * other problems of the group (the same bits alone and in any mix) and agree with spca_solve's
 * for it up to the order of rounding in the contractions and the x-step's sums.  The problems on one
 * matrix (one handle and its clones) whose v = A^T y takes the same plane products share one
 * contraction (a pool): their active starts side by side in one operand, so the matrix is read
 * once per sweep for all of them; a start's sums do not depend on where the others put it.
 * A resident 16-bit handle (SPCA_FP16_RESIDENT) runs every sweep of its problems on its leading
 * planes, as spca_solve does.
 *
 * A group is also a session: problems can be admitted between segments of sweeps while others
 * run (spca_group_admit), and spca_group_step runs the next sweeps of every member, finalising
 * and retiring the members whose starts have all stopped -- continuous batching at sweep
 * boundaries.  Problem i of a call:
 *   h     a handle from spca_create (dense A) on a device with tensor cores, or a clone of one;
 *         read only (several problems and groups may use one handle at once).
 *   prm   as for spca_solve, with lowp_sweeps = 0 (and, on a resident 16-bit handle,
 *         lowp_first = refine_sweeps = 0), total_starts <= r, engine AUTO or TC,
 *         r in 1 .. 65535; timeout_us is not checked; the support gather serves every support
 *         after the first sweep.
 *   x0    r x p starts (host or device per prm.x0_is_device; copied at admission), or NULL for
 *         seeded starts (the same starts as spca_solve with that seed).
 *   res   caller-owned host buffers as for spca_solve, written when the problem finishes; they
 *         must stay valid until then.
 *
 * spca_group_create    a group: its own stream; each call starts after the work queued on
 *                      cuda_stream (as in spca_create).
 * spca_group_destroy   frees it, with any admitted problems (their results are not written);
 *                      NULL is a no-op.
 * spca_group_last_error  static text for the group's last failure ("" if none).
 * spca_group_set_tiles the tile shape of the grouped contraction: tile_n (64 or 128 columns)
 *                      and stages (2..4 for 64, 2..3 for 128); NULL or {0, 0} = chosen when the
 *                      tables are built, from the widest pool (the most starts that share one
 *                      contraction): 64 x 4 up to 64 starts, 128 x 3 above, the shapes bench.py
 *                      --tune measured best for those start counts; a group of resident 16-bit
 *                      matrices only takes 64, 128 or 256 columns by the same widths, 4 stages.
 * spca_group_admit     admit `count` problems (tags[i] identifies problem i in the finished
 *                      lists; NULL = 0 .. count - 1); a member's device memory is allocated here
 *                      (stream-ordered).  On failure none of the call's problems is admitted.
 * spca_group_step      run `sweeps` sweeps of every member (the members admitted since the last
 *                      step begin with their first sweep), then finalise the members whose starts
 *                      have all stopped: their results are written and their tags listed in
 *                      finished[0 .. min(*nfinished, cap)).  Synchronous.
 * spca_group_pending   members admitted and not finished.
 * spca_solve_group     admit the problems, sweep until every start of every problem has stopped
 *                      (the segments captured into CUDA graphs and replayed), write every result;
 *                      the group must have no members.
 * Errors: SPCA_E_INVALID (arguments, a problem's parameters, non-finite x0, an unknown tile shape;
 *         spca_group_last_error says which), SPCA_E_UNSUPPORTED (more than 1024 members),
 *         SPCA_E_BUSY (spca_solve_group on a group with members), SPCA_E_NOMEM, SPCA_E_CUDA,
 *         SPCA_E_TIMEOUT (a bounded device-side wait gave up).
 */
typedef struct spca_group spca_group;
typedef struct {
    spca_handle *h;
    spca_params prm;
    const float *x0;
    spca_result *res;
} spca_problem;
typedef struct {
    int tile_n;
    int stages;
} spca_group_tiles;
int spca_group_create(spca_group **out, void *cuda_stream);
void spca_group_destroy(spca_group *g);
const char *spca_group_last_error(const spca_group *g);
int spca_group_set_tiles(spca_group *g, const spca_group_tiles *tiles);
int spca_group_admit(spca_group *g, spca_problem *probs, int count, const int *tags);
int spca_group_step(spca_group *g, int sweeps, int *finished, int cap, int *nfinished);
int spca_group_pending(const spca_group *g);
int spca_solve_group(spca_group *g, spca_problem *probs, int count, const spca_group_tiles *tiles);

/* spca_destroy -- free the handle's device memory (waits for its stream). NULL is a no-op. */
void spca_destroy(spca_handle *h);

/* spca_strerror -- static text for a status code. */
const char *spca_strerror(int status);

/* spca_last_error -- static text for the last failure of this handle ("" if none). */
const char *spca_last_error(const spca_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* SPCA_H */
