/*
 * sbsolve.h -- C ABI of the shared-LHS batched banded solver for GB300 (sm_103a).
 *
 * The problem (the paper's "single A, multiple b" statement, section 1 and
 * section 2): many tridiagonal or pentadiagonal systems A x_m = b_m, m = 0..M-1,
 * share ONE left-hand-side matrix A.  A is factorised once on the host in FP64
 * (Algorithm 1 for tridiagonal, Algorithm 3 / section 4.1 for pentadiagonal) and a
 * single device copy of its factors is kept; every right-hand side is swept
 * forward and back (Algorithms 2 and 4) in the interleaved layout of Fig. 2.
 *
 * Layout.  A batch of M systems of N unknowns is one array with element (i, m)
 * at index i*ld + m (system index fastest), 0 <= i < N, 0 <= m < M, ld >= M.
 * Columns M <= m < ld are never read or written.
 *
 * Conventions shared by every call.
 *   - Return 0 on success, a negative SB_ERR_* code otherwise; no call throws.
 *     sb_last_error() gives a message for the last failure on this host thread.
 *   - Device pointers must be device (or managed) memory on the device that was
 *     current when the factor was created; the library checks this and rejects
 *     host pointers.  They must be aligned to the element size.
 *   - Solves are asynchronous on `stream` (a cudaStream_t passed as void*, NULL =
 *     the legacy default stream).  The status covers argument checks and the
 *     launch only.
 *   - `x` may be the same pointer as `rhs` (in-place, as in the paper); any
 *     other overlap of the two arrays is rejected.
 *   - A factor handle is immutable once created: it may be used concurrently
 *     from several streams and host threads.  The caller owns every buffer it
 *     passes; the library owns only the factor's device copy.
 */
#ifndef SBSOLVE_H
#define SBSOLVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define SB_OK                0
#define SB_ERR_INVALID_ARG  -1  /* bad size, null or misaligned pointer, host pointer, overlap */
#define SB_ERR_SINGULAR     -2  /* zero or non-finite pivot while factorising (row in message) */
#define SB_ERR_CUDA         -3  /* a CUDA runtime call or kernel launch failed */
#define SB_ERR_ALLOC        -4  /* device or host allocation failed */
#define SB_ERR_UNSUPPORTED  -5  /* valid request this build does not implement */

/* Element type of right-hand sides and solutions in device memory. */
typedef enum { SB_F64 = 0, SB_F32 = 1 } sb_dtype;

/*
 * Arithmetic of a sweep.
 *   SB_ARITH_NATIVE  the storage type's own arithmetic (FP64 for SB_F64, FP32 for
 *                    SB_F32; FP32 when an FP32 right-hand side is solved into an
 *                    FP64 solution).
 *   SB_ARITH_DF32    double-float: each value is the unevaluated sum of two FP32
 *                    numbers (about 48 significant bits, relative rounding about
 *                    2^-47 per operation), computed on the FP32 pipe.  Inputs are
 *                    FP64 (or FP32) and the solution is FP64.  On GB300 the FP64 pipe
 *                    issues 2 operations per clock per SM against 128 for FP32, so
 *                    this mode reaches FP64-level accuracy (1e-13 relative on
 *                    well-conditioned systems) at several times the speed.
 */
typedef enum { SB_ARITH_NATIVE = 0, SB_ARITH_DF32 = 1 } sb_arith;

/* Opaque factor of one shared matrix.  Owns a device copy of the factors. */
typedef struct sb_factor sb_factor;

/*
 * sb_factor_shared_tri -- factorise a shared tridiagonal matrix (section 3.1,
 * Algorithm 1: ch_1 = c_1/b_1; bh_i = b_i - a_i ch_{i-1}, ch_i = c_i/bh_i).
 *
 *   N        number of unknowns, N >= 1.
 *   a, b, c  host arrays of N doubles: sub-diagonal (a[0] ignored), diagonal,
 *            super-diagonal (c[N-1] ignored); row i is a[i] x[i-1] + b[i] x[i]
 *            + c[i] x[i+1].  Read only during the call.
 *   out      receives the new handle (set to NULL on failure).
 *
 * No pivoting (as in the paper): a zero or non-finite pivot bh_i returns
 * SB_ERR_SINGULAR and names the row.  The factors are copied to the current
 * CUDA device; free the handle with sb_factor_destroy.
 */
int sb_factor_shared_tri(int64_t N, const double* a, const double* b, const double* c,
                         sb_factor** out);

/*
 * sb_factor_shared_tri_periodic -- factorise a shared periodic tridiagonal matrix
 * (section 3.3): row i is a[i] x[i-1] + b[i] x[i] + c[i] x[i+1] with the indices
 * taken modulo N, so a[0] multiplies x[N-1] and c[N-1] multiplies x[0] (the corner
 * entries).  As in section 3.3, A = A' + u v^T with u = (-b[0], 0, .., c[N-1]),
 * v = (1, 0, .., -a[0]/b[0]); A' (no corners, b'[0] = 2 b[0], b'[N-1] = b[N-1] +
 * a[0] c[N-1]/b[0]) is factored as by sb_factor_shared_tri and A'^{-1} u is solved
 * once, in FP64 on the host.  Every solve with the handle (sb_solve_batched, _ex,
 * _adjoint, _host, any dtype and arithmetic) returns x = y - f z with y = A'^{-1} b,
 * z = A'^{-1} u and f = (v . y)/(1 + v . z), in one pass over the batch: y_0 is
 * accumulated during the forward sweep and the correction is applied as x is
 * written.  The transpose uses A^T = A'^T + v u^T the same way (no counterpart in
 * the paper).  Refinement and group solves reject periodic handles
 * (SB_ERR_UNSUPPORTED); the partitioned algorithm falls back to the sweeps.
 *   N        >= 3.
 *   a, b, c  host arrays of N doubles, all entries used.
 * SB_ERR_SINGULAR for b[0] = 0, a zero pivot of A' or 1 + v . z = 0.
 */
int sb_factor_shared_tri_periodic(int64_t N, const double* a, const double* b, const double* c,
                                  sb_factor** out);

/*
 * sb_factor_shared_penta_periodic -- factorise a shared cyclic pentadiagonal matrix:
 * row i is a[i] x[i-2] + b[i] x[i-1] + c[i] x[i] + d[i] x[i+1] + e[i] x[i+2] with the
 * indices modulo N (N >= 5), so a[0], a[1], b[0], d[N-1], e[N-2], e[N-1] are corner
 * entries.  Section 5.1's scheme is periodic and the paper refers to the literature
 * for this solve; this library uses the 2 x 2 block form of section 3.3's split:
 * A = A' + U V^T with X = -(top-left 2 x 2 block), U = [X; 0; BL], V = [I; 0;
 * (X^{-1} TR)^T] (TR, BL the corner blocks), A' pentadiagonal (top-left block doubled,
 * bottom-right block minus BL X^{-1} TR, no corners) factored as by
 * sb_factor_shared_penta, and Z = A'^{-1} U and S = I + V^T Z formed once in FP64.
 * Every solve returns x = y - Z S^{-1} V^T y with y = A'^{-1} b in one pass: y_0 and
 * y_1 are accumulated as dot products during the forward sweep, and the first two
 * rows of the backward sweep are held back until the correction is known.  The
 * transpose uses A^T = A'^T + V U^T (no counterpart in the paper).  Refinement and
 * group solves reject periodic handles; the partitioned algorithm falls back to the
 * sweeps.  SB_ERR_SINGULAR for a singular top-left block, a zero pivot of A' or a
 * singular S.
 */
int sb_factor_shared_penta_periodic(int64_t N, const double* a, const double* b, const double* c,
                                    const double* d, const double* e, sb_factor** out);

/*
 * sb_factor_shared_penta -- factorise a shared pentadiagonal matrix A = L R
 * (section 4.1; Algorithm 3 read with the section's equations).
 *
 *   a, b, c, d, e  host arrays of N doubles: the diagonals at offsets -2, -1, 0,
 *                  +1, +2 (row i is a[i] x[i-2] + b[i] x[i-1] + c[i] x[i]
 *                  + d[i] x[i+1] + e[i] x[i+2]); entries that fall outside the
 *                  matrix are ignored.
 * Other arguments and errors as for sb_factor_shared_tri.
 */
int sb_factor_shared_penta(int64_t N, const double* a, const double* b, const double* c,
                           const double* d, const double* e, sb_factor** out);

/* Release a handle and its device memory (NULL is a no-op).  Waits for nothing:
 * the caller must make sure no solve that uses it is still running. */
void sb_factor_destroy(sb_factor* f);

/* Bandwidth (1 = tridiagonal, 2 = pentadiagonal) and N of a handle; returns
 * SB_ERR_INVALID_ARG for a NULL handle or NULL outputs. */
int sb_factor_info(const sb_factor* f, int* half_bandwidth, int64_t* N);

/*
 * sb_solve_batched -- solve A x_m = rhs_m for m = 0..M-1 with the shared factors
 * (forward and backward sweeps of Algorithms 2 and 4), one device pass.
 *
 *   rhs, x   device arrays of N*ld elements of `dtype` in the interleaved layout;
 *            x may equal rhs.
 *   M        number of systems (M = 0 is a no-op), ld >= M the row stride.
 *   dtype    SB_F64: FP64 storage and arithmetic.  SB_F32: FP32 storage and
 *            arithmetic with the FP64 factors rounded to FP32.
 */
int sb_solve_batched(const sb_factor* f, const void* rhs, void* x, int64_t M, int64_t ld,
                     sb_dtype dtype, void* stream);

/*
 * sb_solve_batched_adjoint -- solve A^T y_m = rhs_m with the same factors
 * (no counterpart in the paper: A^T = U^T L^T for A = L U, or R^T L^T for
 * A = L R, swept forward then back).  Arguments as for sb_solve_batched.
 */
int sb_solve_batched_adjoint(const sb_factor* f, const void* rhs, void* x, int64_t M,
                             int64_t ld, sb_dtype dtype, void* stream);

/*
 * sb_solve_batched_ex -- the general form of sb_solve_batched / _adjoint.
 *
 *   transpose  0 solves A x = rhs, 1 solves A^T x = rhs.
 *   rhs_dtype, x_dtype  storage of rhs and x.  Supported combinations:
 *                SB_ARITH_NATIVE: (F64, F64), (F32, F32), (F32, F64);
 *                SB_ARITH_DF32:   (F64, F64), (F32, F64).
 *              Others return SB_ERR_UNSUPPORTED.  x may equal rhs only when the
 *              two dtypes are the same.
 * Other arguments as for sb_solve_batched.
 */
int sb_solve_batched_ex(const sb_factor* f, int transpose, const void* rhs, sb_dtype rhs_dtype,
                        void* x, sb_dtype x_dtype, int64_t M, int64_t ld, sb_arith arith,
                        void* stream);

/*
 * Solve algorithms of a batched solve.
 *   SB_ALGO_SEQUENTIAL   one thread sweeps one system forward then back (Algorithms
 *                        2 and 4 with the interleaved layout of section 2); the
 *                        intermediate of the forward sweep is kept in x.
 *   SB_ALGO_PARTITIONED  this library's own (no counterpart in the paper): a CTA
 *                        keeps a tile of 32 systems on chip (the tile arrives by TMA
 *                        while the previous one is solved), cut into 16 chunks of
 *                        16/32/64 rows (512 threads, one warp per chunk; or 256 threads,
 *                        half a warp per chunk with two systems per thread, the default
 *                        for FP32 rhs) or 32 chunks of 8/16/32 rows (1024 threads);
 *                        every chunk is swept with its own factors and the
 *                        chunks are joined through the small system of their boundary
 *                        values, solved by parallel cyclic reduction (a SPIKE-type
 *                        decomposition, exact up to rounding, whose spikes and reduction
 *                        matrices depend on A only and are computed once, in FP64, with
 *                        the factorisation).  Each rhs element is read once and each x
 *                        element written once.  It applies to FP32 rhs with FP32 or FP64
 *                        x in native arithmetic, 64 <= N <= 1024, rhs 16-byte aligned
 *                        and ld a multiple of 4, when every chunk's factorisation has
 *                        non-zero pivots; elsewhere a solve asked to use it runs the
 *                        sequential sweeps with their default shape.
 *                        With 128-thread CTAs it is the FP64 form for latency-bound
 *                        batches: tiles of 8 systems cut into 16 chunks of 8/16/32 rows
 *                        (32 <= N <= 512), FP64 rhs and x, native arithmetic, the
 *                        boundary system solved by cyclic reduction when every CTA
 *                        has one tile (latency-bound batches), else by block
 *                        Thomas; same fallback.
 *   SB_ALGO_STAGED       the sequential sweeps with both row streams (the rhs in the
 *                        forward sweep, the intermediate in the backward sweep) staged
 *                        through a ring of 8 rows per thread in shared memory by
 *                        cp.async, so the rows in flight take no registers and a CTA
 *                        can run up to 1024 threads (512 in double-float
 *                        arithmetic).  Same arithmetic and results as
 *                        SB_ALGO_SEQUENTIAL; applies to non-periodic factors whose
 *                        coefficients and ring fit in one CTA's shared memory, else
 *                        the sequential sweeps run with their default shape.
 *   SB_ALGO_TWO_ENDED    this library's own: every system is eliminated from its
 *                        first row downwards and from its last row upwards at the
 *                        same time (LU of the top half and of the reversed bottom
 *                        half, computed once in FP64 with the factorisation), the two
 *                        halves meet in a 2P x 2P system whose inverse is precomputed,
 *                        and the back substitution runs outwards from it: two
 *                        independent recurrences per thread and the same FP64
 *                        operations per element, exact up to rounding.  Rows staged
 *                        as in SB_ALGO_STAGED.  Applies to FP64 rhs and x in native
 *                        arithmetic, non-periodic factors, N >= 4 (tridiagonal) or
 *                        N >= 8 (pentadiagonal); elsewhere the sequential sweeps run
 *                        with their default shape.
 */
typedef enum {
  SB_ALGO_SEQUENTIAL = 0,
  SB_ALGO_PARTITIONED = 1,
  SB_ALGO_STAGED = 2,
  SB_ALGO_TWO_ENDED = 3
} sb_algo;

/*
 * Launch shape of a batched solve.
 *   threads             threads per CTA: a multiple of 32 in [32, 512] for
 *                       SB_ALGO_SEQUENTIAL, in [32, 1024] for SB_ALGO_STAGED (at most
 *                       512 in double-float arithmetic) and SB_ALGO_TWO_ENDED; 256
 *                       (16 chunks, two systems per thread),
 *                       512 (16 chunks) or 1024 (32 chunks) for SB_ALGO_PARTITIONED
 *                       with FP32 rhs, 128 for its FP64 form.
 *   ctas_per_sm         cap on resident CTAs per SM (0 = as many as fit; 0 or 1 for
 *                       SB_ALGO_PARTITIONED, which fits one).
 *   systems_per_thread  1 or 2 for SB_ALGO_SEQUENTIAL (each thread interleaves that
 *                       many independent recurrences); 1 for the other algorithms.
 *   algorithm           an sb_algo.
 */
typedef struct {
  int threads;
  int ctas_per_sm;
  int systems_per_thread;
  int algorithm;
} sb_shape;

/* The shape solves with this factor's (half bandwidth, N), arithmetic and dtypes
 * will use: a stored entry if there is one, else the built-in default. */
int sb_shape_get(const sb_factor* f, sb_arith arith, sb_dtype rhs_dtype, sb_dtype x_dtype,
                 sb_shape* out);

/* Store a shape for that key (process-wide, on the factor's device); for example
 * one loaded from a tuning cache.  SB_ERR_INVALID_ARG for an out-of-range shape. */
int sb_shape_set(const sb_factor* f, sb_arith arith, sb_dtype rhs_dtype, sb_dtype x_dtype,
                 const sb_shape* shape);

/*
 * sb_autotune -- time every candidate shape (sequential: threads 64..512, CTAs/SM
 * 0..2, systems per thread 1..2; partitioned, where it applies) on the caller's buffers with CUDA events (one warm-up
 * and the best of three launches each), store the fastest as for sb_shape_set and
 * return it in *best (and its time in *best_ms; either may be NULL).  x is
 * overwritten and must differ from rhs; arguments otherwise as for
 * sb_solve_batched_ex.  Blocking: it synchronises on `stream`.  The autotuner is
 * this library's own (the paper's kernels have a fixed one-thread-per-system shape).
 */
int sb_autotune(const sb_factor* f, int transpose, const void* rhs, sb_dtype rhs_dtype, void* x,
                sb_dtype x_dtype, int64_t M, int64_t ld, sb_arith arith, void* stream,
                sb_shape* best, float* best_ms);

/*
 * Shared matrices of the finite-difference workloads (sections 3.2, 4.2 and 5.1).
 * Each is I + coef * K for an operator K:
 *   SB_MAT_DIFFUSION_DIRICHLET  K = tridiag(-1, 2, -1) with the stencil truncated at
 *                               the first and last rows (backward-Euler / left-hand
 *                               side of section 3.2's scheme); tridiagonal.
 *   SB_MAT_HYPER_HINGED         K = D2 * D2 with D2 = tridiag(1, -2, 1) truncated:
 *                               interior rows (1, -4, 6, -4, 1) of section 4.2,
 *                               first/last rows (5, -4, 1), (-4, 6, -4, 1).
 *   SB_MAT_HYPER_TRUNCATED      K = Toeplitz (1, -4, 6, -4, 1) cut at the edges.
 *   SB_MAT_CH_NOFLUX            K = D2N * D2N with the cell-centred Neumann
 *                               D2N = rows (-1, 1), (1, -2, 1), ..., (1, -1): the
 *                               implicit matrix of section 5.1 with no-flux ends
 *                               (coef = dt * gamma in grid units).
 *   SB_MAT_DIFFUSION_PERIODIC   K = tridiag(-1, 2, -1) wrapping around (section 3.3's
 *                               matrix; N >= 3): a[0] and c[N-1] are the corner
 *                               entries; factor it with sb_factor_shared_tri_periodic.
 *   SB_MAT_CH_PERIODIC          K = D2P * D2P, rows (1, -4, 6, -4, 1) wrapping around:
 *                               section 5.1's implicit matrix with the paper's periodic
 *                               ends (N >= 5); factor it with
 *                               sb_factor_shared_penta_periodic.
 * `diags` is a host array of (2P+1)*N doubles (P = 1 for the diffusion matrices, 2
 * otherwise), diagonal-major: diags[k*N + i] is row i of the diagonal at offset
 * k - P; entries outside the matrix are written as 0 (except the periodic
 * corners).  Host only; no GPU needed.
 * Returns SB_ERR_INVALID_ARG for an unknown kind, N < 1, a NULL or non-finite input.
 */
#define SB_MAT_DIFFUSION_DIRICHLET 1
#define SB_MAT_HYPER_HINGED        2
#define SB_MAT_HYPER_TRUNCATED     3
#define SB_MAT_CH_NOFLUX           4
#define SB_MAT_DIFFUSION_PERIODIC  5
#define SB_MAT_CH_PERIODIC         6
int sb_build_matrix(int kind, int64_t N, double coef, double* diags);

/*
 * sb_solve_batched_host -- sb_solve_batched_ex for a batch held in host memory.
 * The batch is cut into chunks of chunk_systems systems (0 = about eight chunks);
 * each chunk is copied to the device, solved and copied back on one of three
 * internal streams, so both copy directions overlap the solves of neighbouring
 * chunks.  Asynchronous: the work is ordered after prior work on `stream` and
 * `stream` waits for all of it (synchronise it before reading x_host).
 *   rhs_host, x_host  host arrays in the N x ld interleaved layout (may be the same
 *                     array); page-locked memory is needed for the copies to overlap.
 *   work              caller-owned device workspace of sb_host_workspace_bytes() bytes.
 * Other arguments and the supported dtype/arith combinations as for
 * sb_solve_batched_ex.  (No counterpart in the paper, whose batches live on the GPU.)
 */
int sb_host_workspace_bytes(const sb_factor* f, int64_t M, int64_t chunk_systems,
                            sb_dtype rhs_dtype, sb_dtype x_dtype, size_t* bytes);
int sb_solve_batched_host(const sb_factor* f, int transpose, const void* rhs_host,
                          sb_dtype rhs_dtype, void* x_host, sb_dtype x_dtype, int64_t M,
                          int64_t ld, sb_arith arith, int64_t chunk_systems, void* work,
                          size_t work_bytes, void* stream);

/*
 * Mixed precision with iterative refinement (no counterpart in the paper, which
 * does not discuss precision; the sweeps are those of sections 3.1 and 4.1): FP32
 * storage of the right-hand sides, FP32 sweeps with the FP64 factors rounded to
 * FP32, and n_refine correction passes  r = b - A x,  d = A_32^{-1} r,  x += d
 * whose residual uses A's FP64 entries, evaluated in FP64 (residual_arith =
 * SB_ARITH_NATIVE) or double-float (SB_ARITH_DF32).  The solution is FP64.
 *
 *   rhs        device FP32, N x ld interleaved;  x  device FP64, same layout
 *              (must not overlap rhs).
 *   n_refine   0..16 correction passes (0 = plain FP32 solve into FP64).
 *   work       device workspace of sb_refine_workspace_bytes() bytes (FP32, one
 *              element per solution element), owned by the caller; unused when
 *              n_refine == 0 (may be NULL then).  Its contents are scratch.
 * One kernel runs every pass of a tile of 32 systems before its next tile.  The
 * residual of a pass is built from a window of x inside the backward sweep of the
 * pass before it, with the passes eliminating alternately from the top (A = LU)
 * and from the bottom (the factors of the row- and column-reversed matrix, made
 * once at factor time); where those factors or the shared memory they need are
 * missing, each pass runs its own forward and backward sweeps in the same kernel.
 * The result does not depend on the launch shape beyond rounding.
 */
int sb_refine_workspace_bytes(const sb_factor* f, int64_t M, int64_t ld, size_t* bytes);
int sb_solve_batched_refined(const sb_factor* f, const float* rhs, double* x, int64_t M,
                             int64_t ld, int n_refine, sb_arith residual_arith, void* work,
                             size_t work_bytes, void* stream);

/*
 * sb_solve_batched_refined_noalloc -- sb_solve_batched_refined for callers that
 * cannot allocate device memory when they solve (code inside a framework whose
 * memory pool owns all allocations, allocation-free real-time loops, C callers
 * without an allocator).  It takes no workspace and allocates nothing: its FP32
 * scratch is a 16 MiB array compiled into the library, which every GPU that
 * loads the library keeps until the process exits.  The paper has no
 * counterpart; this is a convenience of this library.
 *
 *   Limit: (N - 1) * ld + M <= 4194304 elements (4 Mi FP32 values), otherwise
 *          SB_ERR_INVALID_ARG with a message; other arguments and results as for
 *          sb_solve_batched_refined.
 *   The first call on each device looks up the scratch array's device address
 *   (and sets up the kernels); make that first call before any stream capture.
 *   All calls share the one scratch array: calls that overlap on the GPU (other
 *   streams, other host threads) race on it and must be serialised by the caller.
 */
int sb_solve_batched_refined_noalloc(const sb_factor* f, const float* rhs, double* x, int64_t M,
                                     int64_t ld, int n_refine, sb_arith residual_arith,
                                     void* stream);

/*
 * sb_solve_batched_groups -- solve G (1..8) independent shared-LHS groups, each
 * with its own factor (its own N) and batch, with one kernel launch per pass:
 * the persistent CTAs are divided between the groups in proportion to N*M and
 * each stages its own group's factors.  All factors of one call must have the
 * same bandwidth and live on one device.
 *   f, rhs, x, M, ld, work, work_bytes   arrays of G entries (work/work_bytes only
 *                                        when n_refine > 0; may be NULL otherwise).
 *   rhs_dtype, x_dtype, arith            as for sb_solve_batched_ex (n_refine == 0);
 *                                        with n_refine > 0 rhs_dtype is SB_F32 or
 *                                        SB_F64 (an FP64 right-hand side is rounded
 *                                        to FP32 for the sweeps and used in FP64 by
 *                                        the residual), x_dtype SB_F64 and arith
 *                                        SB_ARITH_NATIVE (FP32 sweeps).
 *   residual_arith                       as for sb_solve_batched_refined.
 * Launches: one per call, whatever G and n_refine are.
 */
int sb_solve_batched_groups(int G, const sb_factor* const* f, const void* const* rhs,
                            void* const* x, const int64_t* M, const int64_t* ld,
                            sb_dtype rhs_dtype, sb_dtype x_dtype, sb_arith arith, int n_refine,
                            sb_arith residual_arith, void* const* work, const size_t* work_bytes,
                            void* stream);

/*
 * Implicit time steppers with a shared matrix (sections 3.2, 4.2 and 5.1), each
 * step one fused kernel, runs of steps replayed as CUDA graphs.
 * One step solves  A C^{n+1} = B C^n + E (C^3 - C)^n  for every simulation:
 *   SB_STEP_DIFFUSION      A = I + coef K, K = tridiag(-1, 2, -1) with Dirichlet rows.
 *                          SB_SCHEME_BE: B = I (backward Euler, coef = r = dt/dx^2);
 *                          SB_SCHEME_CN: B = I - coef K (section 3.2's Crank-Nicolson,
 *                          coef = sigma = dt/(2 dx^2)).  bc SB_BC_DIRICHLET, or
 *                          SB_BC_PERIODIC (the paper's own ends, sections 3.2-3.3:
 *                          K wraps around, A is factored as by
 *                          sb_factor_shared_tri_periodic and every step applies the
 *                          Sherman-Morrison correction inside the fused kernel).
 *   SB_STEP_HYPERDIFFUSION A = I + coef D4 with bc SB_BC_HINGED (D4 = D2 D2),
 *                          SB_BC_TRUNCATED (Toeplitz 1,-4,6,-4,1) or SB_BC_PERIODIC
 *                          (D4 = D2P D2P wrapping around, N >= 5, the cyclic
 *                          pentadiagonal solve of sb_factor_shared_penta_periodic);
 *                          B = I (BE) or I - coef D4 (section 4.2's Crank-Nicolson).
 *   SB_STEP_CAHN_HILLIARD  section 5.1's semi-implicit scheme (scheme SB_SCHEME_BE):
 *                          A = I + dt coef D4, B = I, E = dt D2, with coef = gamma in
 *                          grid units (dx = 1); bc SB_BC_NOFLUX (D2 = D2_N, D4 = D2_N^2)
 *                          or SB_BC_PERIODIC (the paper's own ends: D2_P, D4_P, N >= 5).
 * The stepper owns the factorised A and the right-hand-side coefficients.
 */
typedef struct sb_stepper sb_stepper;
#define SB_STEP_DIFFUSION      1
#define SB_STEP_HYPERDIFFUSION 2
#define SB_STEP_CAHN_HILLIARD  3
#define SB_SCHEME_BE 0
#define SB_SCHEME_CN 1
#define SB_BC_DIRICHLET 0
#define SB_BC_HINGED    1
#define SB_BC_TRUNCATED 2
#define SB_BC_NOFLUX    3
#define SB_BC_PERIODIC  4
/* run modes: fused step kernel replayed from a captured CUDA graph (64 steps per
 * graph; falls back to direct launches on the legacy NULL stream or while the
 * stream is being captured), fused kernel launched directly, or the unfused
 * reference pipeline (a separate right-hand-side kernel into `work`, then the
 * batched solve) that mirrors the paper's two-kernel step. */
#define SB_RUN_GRAPH   0
#define SB_RUN_DIRECT  1
#define SB_RUN_UNFUSED 2

int sb_stepper_create(int kind, int scheme, int bc, int64_t N, double coef, double dt,
                      sb_stepper** out);
void sb_stepper_destroy(sb_stepper* st);
/* The stepper's factor of A (owned by the stepper; valid until it is destroyed). */
const sb_factor* sb_stepper_factor(const sb_stepper* st);
/* Bytes of device workspace SB_RUN_UNFUSED needs for a (M, ld) batch. */
int sb_stepper_workspace_bytes(const sb_stepper* st, int64_t M, int64_t ld, size_t* bytes);
/*
 * sb_stepper_run -- advance `state` (device FP64, N x ld interleaved, M simulations)
 * by nsteps steps in place, asynchronously on `stream`.  arith as for
 * sb_solve_batched_ex.  `work`/`work_bytes` are used only by SB_RUN_UNFUSED (the
 * caller owns the workspace; NULL otherwise).  The first SB_RUN_GRAPH call for a
 * given (state, M, ld, arith) captures and caches a graph: make that first call
 * outside any stream capture of the caller's own.
 */
int sb_stepper_run(sb_stepper* st, double* state, int64_t M, int64_t ld, sb_arith arith,
                   int64_t nsteps, int mode, void* work, size_t work_bytes, void* stream);

/*
 * sb_stepper_run_refined -- nsteps steps with FP32 sweeps and iterative refinement
 * (the precision pattern of sb_solve_batched_refined applied to a time step): each
 * step builds its right-hand side f in FP64 (one kernel, as the unfused step), then
 * solves A C^{n+1} = f by an FP32 sweep of f rounded to FP32 into the FP64 state and
 * n_refine passes r = f - A C (FP64 or double-float residual, residual_arith),
 * d = A_32^{-1} r, C += d; 64-step CUDA graphs in SB_RUN_GRAPH mode.
 *   state   device FP64, N x ld; work: sb_stepper_refined_workspace_bytes() bytes
 *           of device memory (the FP64 f and the FP32 scratch), caller-owned.
 * Non-periodic steppers only (SB_ERR_UNSUPPORTED otherwise); a forced stepper is
 * rejected.  Other arguments as for sb_stepper_run.
 */
int sb_stepper_refined_workspace_bytes(const sb_stepper* st, int64_t M, int64_t ld, size_t* bytes);
int sb_stepper_run_refined(sb_stepper* st, double* state, int64_t M, int64_t ld, int n_refine,
                           sb_arith residual_arith, int64_t nsteps, int mode, void* work,
                           size_t work_bytes, void* stream);

/*
 * sb_stepper_set_forcing -- turn a periodic Cahn-Hilliard stepper into the
 * travelling-wave forced scheme of section 6.1 (the forced equation written in the
 * frame of the wave, eta = x - v t), in grid units:
 *   (I + sigma D4_P) C^{n+1} = C^n + alpha D2_P (C^3 - C)^n + adv W(C^n) + amp_m g_i
 * W is the fifth-order Hamilton-Jacobi WENO derivative (the scheme the paper takes
 * from Osher and Fedkiw's book, i.e. Jiang and Peng's), biased toward lower rows
 * (rows i-3..i+2) for adv >= 0 and toward higher rows for adv < 0;
 * adv = dt v / dx; g (host, N doubles, copied) is the forcing profile, for the paper
 * g_i = dt k cos(k eta_i); amp_m (per system, given to sb_stepper_run_forced) is the
 * forcing amplitude f_0 of simulation m.  May be called again to change adv or g.
 * Native FP64 only.  SB_ERR_UNSUPPORTED for other steppers; SB_ERR_INVALID_ARG for
 * NULL or non-finite input.  Synchronises the device.
 */
int sb_stepper_set_forcing(sb_stepper* st, double adv, const double* g);

/*
 * sb_stepper_run_forced -- nsteps forced steps of `state` in place (one fused kernel
 * per step: the right-hand side, WENO term and forcing built inside the forward
 * sweep; graph-captured in SB_RUN_GRAPH mode).  amp: device array of M doubles.
 * A forced stepper runs only through this call (sb_stepper_run, the coarsening run
 * and the rollouts reject it).  Other arguments as for sb_stepper_run.
 */
int sb_stepper_run_forced(sb_stepper* st, double* state, const double* amp, int64_t M, int64_t ld,
                          int64_t nsteps, int mode, void* stream);

/*
 * sb_stepper_run_coarsening -- nsteps fused Cahn-Hilliard steps (as
 * sb_stepper_run with SB_RUN_DIRECT) that also record section 5.3's typical domain
 * size after every step: ell[n] = mean over the M systems of 1 / (1 - <C^2>), with
 * <C^2> the mean of C_i^2 over the N grid points (the periodic rectangle rule for
 * (1/L) int C^2 dx) of the state after step n + 1.  Each system's value is formed in
 * the step's backward sweep; the mean is a fixed-order reduction, so ell is the
 * same on every run.
 *   st     a SB_STEP_CAHN_HILLIARD stepper (SB_BC_NOFLUX or SB_BC_PERIODIC).
 *   ell    device array of nsteps doubles.
 *   work   device workspace of (M + 256) doubles.
 * Other arguments as for sb_stepper_run.  SB_ERR_UNSUPPORTED for other stepper kinds.
 */
int sb_stepper_run_coarsening(sb_stepper* st, double* state, int64_t M, int64_t ld, sb_arith arith,
                              int64_t nsteps, double* ell, void* work, size_t work_bytes,
                              void* stream);

/*
 * Differentiable rollouts (no counterpart in the paper,
 * which only runs forward).  For a backward-Euler diffusion / hyperdiffusion or a
 * Cahn-Hilliard stepper, the rollout x_{n+1} = A(p)^{-1} F(x_n), n < nsteps, with p
 * the stepper's coefficient (r, or gamma), and a loss L(x_T) chosen by the caller:
 *
 *   sb_rollout_forward   x_T from x_0 = C0, keeping a checkpoint every ckpt_every
 *                        steps in `work`.
 *   sb_rollout_backward  from grad_CT = dL/dx_T: grad_C0 = dL/dx_0, and dL/dp per
 *                        system (M doubles, optional) and summed over the batch
 *                        (one double, optional; a fixed-order sum, so repeatable).
 *                        Recomputes each segment from its checkpoint (bitwise the
 *                        forward states), then per step one fused kernel:
 *                        mu = A^{-T} gbar (same factors), dL/dp -= mu.(dA/dp)x_{n+1},
 *                        gbar <- J_F(x_n)^T mu.  The adjoint arithmetic is FP64;
 *                        `arith` selects the arithmetic of the recomputed steps and
 *                        must match the forward call.
 *
 * All arrays are device FP64 in the N x ld interleaved layout (grad outputs must
 * not overlap `work`).  `work` is caller-owned, sb_rollout_workspace_bytes() bytes:
 * (ceil(nsteps/ckpt_every) + ckpt_every + 2) states of N*ld doubles plus M + 256
 * doubles.  The same work buffer (unchanged between the calls), sizes, nsteps,
 * ckpt_every and arith must be passed to the forward and backward calls.
 * Crank-Nicolson steppers return SB_ERR_UNSUPPORTED.
 */
int sb_rollout_workspace_bytes(const sb_stepper* st, int64_t M, int64_t ld, int64_t nsteps,
                               int64_t ckpt_every, size_t* bytes);
int sb_rollout_forward(sb_stepper* st, const double* C0, double* CT, int64_t M, int64_t ld,
                       int64_t nsteps, int64_t ckpt_every, sb_arith arith, void* work,
                       size_t work_bytes, void* stream);
int sb_rollout_backward(sb_stepper* st, const double* grad_CT, double* grad_C0,
                        double* grad_param_per_system, double* grad_param, int64_t M, int64_t ld,
                        int64_t nsteps, int64_t ckpt_every, sb_arith arith, void* work,
                        size_t work_bytes, void* stream);

/*
 * sb_device_timeouts -- the number of CTAs of SB_ALGO_PARTITIONED solves on `device`
 * that gave up waiting for a tile copy since the previous call (the count is then
 * reset to 0).  Every wait in those kernels is bounded; a CTA that gives up leaves
 * the rest of its tiles unwritten, so a non-zero count means the outputs of the
 * launches since the previous call are incomplete.  Synchronous (device-wide).
 * SB_ERR_INVALID_ARG for a NULL count, SB_ERR_CUDA on a CUDA error.
 */
int sb_device_timeouts(int device, unsigned* count);

/* Message for the last failed call on this host thread ("" if none). */
const char* sb_last_error(void);

/* Library version string. */
const char* sb_version(void);

/*
 * sb_measure_rates -- arithmetic throughputs of `device`, measured: FP64 fused
 * multiply-adds per second (each 2 flop), FP32 fused multiply-adds per second and
 * FP64 -> FP32 -> FP64 conversions per second (each pair counted as two).  Each is
 * timed with CUDA events on many independent dependency chains per thread over a
 * grid that fills every SM (middle of three launches after a warm-up), so it is
 * the pipe's rate.  These are the ceilings the solver's FP64-bound kernels are
 * reported against (this library's own measurement; no counterpart in the paper).
 * Blocking; allocates and frees a small device buffer.  SB_ERR_INVALID_ARG for a
 * NULL result, SB_ERR_CUDA on a CUDA error.
 */
typedef struct {
  double fp64_fma_per_s;
  double fp32_fma_per_s;
  double f64_f32_conversions_per_s;
  int sm_count;
} sb_rates;
int sb_measure_rates(int device, sb_rates* out);

#ifdef __cplusplus
}
#endif

#endif /* SBSOLVE_H */
