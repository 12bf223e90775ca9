/*
 * ebv.h -- C ABI of the GB300 (sm_103a) Equal bi-Vectorized LU solver.
 *
 * The method (Hashemi, Lahooti, Shirani, "Equal bi-Vectorized (EbV) method to
 * high performance on GPU", arXiv 1907.05767):
 *   - Eq. 1:  AX = B  <=>  L(UX) = B.  Factor A = LU, solve LY = B by forward
 *             substitution, then UX = Y by backward substitution.
 *   - Eq. 2:  A is diagonally dominant, so no pivoting is needed.
 *   - Eq. 6a-c: Doolittle elimination.  Step r divides the L vector (column r
 *             below the pivot) by the pivot A_rr and subtracts the outer product
 *             of the L and U vectors from the trailing matrix.
 *   - Eq. 7a-e: the 2n vectors (n columns of L, n rows of U) are paired long
 *             with short so that every thread gets the same amount of work.
 *   - Eq. 4c: A^{-1} as the product of the elimination's elementary
 *             transformations, U^{-1} L^{-1} (ebv_inverse).
 *
 * Conventions shared by every entry point
 *   - Matrices are row-major: element (i, j) of a dense matrix is at
 *     a[i*ld + j], ld >= n.  A band matrix with kl sub- and ku super-diagonals
 *     is stored as a "row band": a_ij at ab[i*ld + (j - i + kl)] for
 *     i - kl <= j <= i + ku, ld >= kl + ku + 1 (other slots are ignored).
 *     Right-hand sides B are n x nrhs row-major with leading dimension ldb.
 *   - Factors are returned packed in place ("L\U"): the strict lower triangle
 *     holds L (its unit diagonal is implied), the upper triangle with the
 *     diagonal holds U.
 *   - Every pointer documented "device" must point to device memory of the
 *     current CUDA device; the caller owns all memory.  The library never
 *     allocates or frees device memory, never synchronises the host inside a
 *     call, and issues all work on `stream` (a cudaStream_t, NULL = legacy
 *     default stream), so the calls are stream-ordered and can be captured
 *     into a CUDA graph.
 *   - Invalid arguments are reported synchronously (EBV_ERR_ARG) before any
 *     work is enqueued.  A failed kernel launch returns EBV_ERR_CUDA.
 *     Numerical trouble is reported through device-side `info` words,
 *     LAPACK-style: 0 = fine, k > 0 = the first pivot that was zero or not
 *     finite is U(k-1, k-1) (1-based k).  The elimination still runs to the
 *     end (results are then meaningless but the call stays well-defined).
 *   - Device-side waits inside the library's kernels are bounded; on expiry a
 *     kernel sets EBV_ERR_TIMEOUT in its status word and returns.
 *   - Calls are reentrant; concurrent calls must use distinct workspaces.
 *   - One device per process: the library prepares each kernel once per
 *     process, on the device current at its first use (shared-memory limits,
 *     occupancy and SM counts), as one process per GPU does.  On another
 *     device those settings are missing and a launch that needs them fails
 *     (EBV_ERR_CUDA).
 */
#ifndef EBV_H_
#define EBV_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define EBV_API __attribute__((visibility("default")))
#else
#define EBV_API
#endif

typedef void *ebv_stream_t; /* a cudaStream_t */

typedef enum {
  EBV_OK = 0,
  EBV_ERR_ARG = 1,           /* invalid argument (sizes, null pointer, alignment, precision) */
  EBV_ERR_ZERO_PIVOT = 2,    /* a zero pivot (reported through info) */
  EBV_ERR_NONFINITE = 3,     /* a non-finite pivot (reported through info) */
  EBV_ERR_NOT_CONVERGED = 4, /* refinement stopped at max_iter above tol */
  EBV_ERR_TIMEOUT = 5,       /* a bounded device wait expired */
  EBV_ERR_CUDA = 6,          /* a CUDA runtime/driver call failed */
  EBV_ERR_UNSUPPORTED = 7,   /* valid but not implemented combination */
  EBV_ERR_WORKSPACE = 8      /* workspace missing or smaller than ebv_workspace_size() */
} ebv_status_t;

typedef enum {
  EBV_FP64 = 0,       /* binary64 throughout */
  EBV_FP32 = 1,       /* binary32 throughout */
  EBV_MIXED_BF16 = 2, /* FP32 factors whose trailing updates take bfloat16
                         operands on the tensor cores (FP32 accumulation);
                         FP64 for the refinement's residual r = b - Ax and
                         update x += d, and for the pivot reciprocals (formed
                         as 1/(double)a_rr, rounded once to binary32 for the
                         FP32 factors; EBV_FP32 does the same) */
  EBV_MIXED_FP16 = 3  /* as above with IEEE half operands, each operand panel
                         scaled by a power of two to stay in half's normal range */
} ebv_prec_t;

/*
 * EBV_BAND_SYM: a symmetric A in the same row-band storage as EBV_BAND with
 * kl == ku (both halves present).  The factorisation uses the lower half:
 * for symmetric A the U vectors are the scaled L vectors, U12 = D11 L21^T
 * with D11 the pivots (eq. 6a-b scale both vectors by the same pivot), and
 * the trailing update L21 D11 L21^T is symmetric, so only its block-lower
 * part is formed; the upper half of the array is read by nothing and is
 * written once at the end with U = D L^T.  The result is the same packed L\U
 * band as EBV_BAND and ebv_solve treats both alike.  (Project addition: the LDL^T reading of the
 * method for symmetric diagonally dominant systems.)
 */
/*
 * EBV_BAND_SYM_LOWER: a symmetric A stored as the lower half of its band
 * only, kl + 1 entries per row: a_ij at ab[i*ld + (j - i + kl)] for
 * i - kl <= j <= i, ld >= kl + 1, ku == kl (half the memory of EBV_BAND_SYM).
 * ebv_factor leaves the LDL^T form in the same array: L strictly below the
 * diagonal (unit diagonal implied) and the pivots d_i = u_ii on it, since
 * U = D L^T.  ebv_solve takes the factors in that storage.  (Project
 * addition, the LDL^T reading of Eq. 6a-b with both its flops and its
 * storage halved.)
 */
/*
 * EBV_PROFILE: a matrix whose band width varies row by row (a profile, or
 * skyline, matrix; the sparse case of the paper's first experiment read as
 * an uneven band) stored compactly by 64-blocks: row block b keeps columns
 * lo[b] .. 64b+63 of its 64 rows (its lower part with the whole diagonal
 * block), column block c keeps rows up[c] .. 64c-1 of its 64 columns (its
 * part above the diagonal block), each row-major.  The buffer holds, for
 * nb = ceil(n/64) blocks, int32 lo[nb], int32 up[nb], int64 offL[nb],
 * int64 offU[nb] (element offsets of the two parts) and, from byte
 * align256(24 nb), the values (double or float).  ebv_profile_from_band
 * builds it from a row band.  desc->kl / ku must bound the profile (the
 * values ebv_profile_from_band returns); ld is ignored.  No row exchanges,
 * so fill stays inside the profile and ebv_factor overwrites the values by
 * the packed factors in place; ebv_solve takes them in the same buffer.
 * EBV_FP64 and EBV_FP32 only; a band whose few wide rows would make band
 * storage pay their width on every row stores only its profile.
 */
/*
 * EBV_DENSE_SYM: a symmetric dense A, row-major with ld >= n, of which only
 * the lower triangle (a_ij, j <= i) is read; the entries above the diagonal
 * are never read nor written.  ebv_factor leaves the LDL^T form in the lower
 * triangle (L strictly below the diagonal, unit diagonal implied, the pivots
 * d_i = u_ii on it; U = D L^T, Eq. 6a-b), forming only the block-lower part
 * of each trailing update: n^3/3 flops instead of 2n^3/3.  ebv_solve takes the
 * factors in that storage (refinement, FP64 only, reads A's lower triangle
 * from a_orig).  EBV_FP64 and EBV_FP32; the mixed precisions return
 * EBV_ERR_UNSUPPORTED, as do ebv_inverse and ebv_gesv_host.  desc->kl / ku
 * are ignored.  (Project addition: the dense form of the symmetric mode.)
 */
typedef enum {
  EBV_DENSE = 0,
  EBV_BAND = 1,
  EBV_BAND_SYM = 2,
  EBV_BAND_SYM_LOWER = 3,
  EBV_PROFILE = 4,
  EBV_DENSE_SYM = 5
} ebv_storage_t;

typedef struct ebv_desc {
  int64_t n;       /* order of A, n >= 0 */
  int64_t ld;      /* row stride in elements (dense: >= n; band: >= kl+ku+1; lower half: >= kl+1) */
  int64_t kl, ku;  /* band widths, 0 <= kl, ku < n (ignored for EBV_DENSE and EBV_DENSE_SYM) */
  int32_t storage; /* ebv_storage_t */
  int32_t reserved;
} ebv_desc_t;

typedef struct ebv_refine {
  double tol;       /* stop when max_c ||b_c - A x_c||_inf / ||b_c||_inf <= tol */
  int32_t max_iter; /* upper bound on residual evaluations after the first solve */
  int32_t reserved;
} ebv_refine_t;

/* Written by the device at the end of a refined solve. */
typedef struct ebv_refine_report {
  int32_t iters;       /* corrections applied after the initial solve */
  int32_t status;      /* EBV_OK, or EBV_ERR_NOT_CONVERGED */
  double resid_first;  /* relative residual of the initial (unrefined) solution */
  double resid_final;  /* relative residual of the returned solution */
} ebv_refine_report_t;

/* Library version, as 10000*major + 100*minor + patch. */
EBV_API int32_t ebv_version(void);

/* Human-readable name of a status code (static storage). */
EBV_API const char *ebv_status_string(ebv_status_t s);

/*
 * Bytes of device workspace that ebv_factor / ebv_solve need for this matrix,
 * precision and number of right-hand sides (the same buffer may serve both,
 * one call at a time).  Returns 0 for invalid arguments or when none is needed.
 */
EBV_API size_t ebv_workspace_size(const ebv_desc_t *desc, ebv_prec_t prec, int64_t nrhs);

/*
 * ebv_factor -- A = LU without pivoting (Eq. 6a-c, equalised as in Eq. 7).
 *
 *   desc      matrix shape and storage.
 *   prec      EBV_FP64 or EBV_FP32: `a` (device, double* or float*) is
 *             overwritten by the packed factors; `lowp` must be NULL.
 *             EBV_MIXED_BF16 / EBV_MIXED_FP16: `a` is a device double*
 *             holding A and is NOT modified; `lowp` (device float*) receives
 *             the packed FP32 factors.  Dense: lowp is n x n, leading
 *             dimension n, and the trailing (Schur) updates are computed from
 *             bfloat16 / half operands on the tensor cores with FP32
 *             accumulation.  Band: lowp has the band layout of `a` (n rows of
 *             ld floats) and the updates run in FP32 (a band's updates are
 *             too thin for the tensor cores); ebv_solve with `refine` then
 *             brings X to FP64 accuracy.
 *   info_dev  device int32: 0, or the 1-based index of the first zero or
 *             non-finite pivot.  Always written.
 *   ws        device workspace of ws_bytes >= ebv_workspace_size(desc, prec, 0),
 *             256-byte aligned (may be NULL when that size is 0).
 * FP64 factorisations that run as 64-column panels (the band, symmetric and
 * profile storages, and dense systems of order <= 256) overlap work on two
 * internal side streams of the device: the rest of each panel's trailing
 * update beside the next panel's diagonal block (symmetric storages past two
 * panels, the others past four) and, without symmetry, each panel's U12
 * beside its L21.  They are forked from and joined back to `stream` inside
 * the call (so the call stays stream-ordered and capturable); the first such
 * call on a device creates those streams and their events: make it before
 * any stream capture.
 * Band storage (EBV_BAND, EBV_BAND_SYM, EBV_BAND_SYM_LOWER) supports every precision (the mixed ones as above);
 * fill-in stays inside the band because no rows are exchanged.  A band whose width varies row by row
 * (a profile, or skyline, matrix stored in its widest band) costs the work of
 * its profile: the factorisation first finds each 64-block's envelope and
 * skips the tiles outside it (see ebv_debug_set_band_envelope).
 * Returns EBV_ERR_ARG for an invalid descriptor or precision, a null or
 * misaligned pointer (a, info_dev, lowp for the mixed precisions, ws; the
 * profile buffer 256-byte aligned); EBV_ERR_UNSUPPORTED for the mixed
 * precisions with EBV_PROFILE or EBV_DENSE_SYM; EBV_ERR_WORKSPACE for a
 * missing or short ws; EBV_ERR_CUDA when a launch fails.  All but the last
 * are returned before anything is enqueued.
 */
EBV_API ebv_status_t ebv_factor(const ebv_desc_t *desc, ebv_prec_t prec, void *a, void *lowp,
                        int32_t *info_dev, void *ws, size_t ws_bytes, ebv_stream_t stream);

/*
 * ebv_solve -- X = A^{-1} B from the factors: LY = B, then UX = Y (Eq. 1).
 *
 *   lu        device: packed factors from ebv_factor (double* for EBV_FP64,
 *             float* for EBV_FP32 and the mixed precisions, i.e. `lowp`).
 *   a_orig    device double*, the original A (same desc); required whenever
 *             `refine` is given (it is the A of the FP64 residual) and ignored
 *             otherwise (may be NULL).
 *   b         device, n x nrhs, leading dimension ldb >= nrhs; overwritten by X.
 *             double* for EBV_FP64 and the mixed precisions, float* for EBV_FP32.
 *   refine    NULL: no refinement.  Otherwise iterative refinement: r = b - A x
 *             in FP64, correction from the factors, x += d in FP64, until the
 *             relative residual (max over columns of ||r||_inf / ||b||_inf) is
 *             <= tol or max_iter residuals were taken.  The stop test runs on
 *             the device (no host synchronisation).
 *   report_dev device ebv_refine_report_t, written when refine != NULL (may be
 *             NULL otherwise).
 *   ws        workspace of ws_bytes >= ebv_workspace_size(desc, prec, nrhs).
 * Returns EBV_ERR_ARG for an invalid descriptor or precision, nrhs outside
 * 0..2^20, ldb < nrhs, a null or misaligned pointer, or refine with a
 * negative or NaN tol or max_iter outside 0..1000; EBV_ERR_UNSUPPORTED for
 * refine with EBV_FP32 (refinement returns FP64 solutions) and for the mixed
 * precisions with EBV_PROFILE or EBV_DENSE_SYM; EBV_ERR_WORKSPACE for a
 * missing or short ws; EBV_ERR_CUDA when a launch fails.  The outcome of the
 * refinement is in report_dev (EBV_ERR_NOT_CONVERGED there), on the device.
 */
EBV_API ebv_status_t ebv_solve(const ebv_desc_t *desc, ebv_prec_t prec, const void *lu, const double *a_orig,
                       void *b, int64_t nrhs, int64_t ldb, const ebv_refine_t *refine,
                       ebv_refine_report_t *report_dev, void *ws, size_t ws_bytes, ebv_stream_t stream);

/*
 * Batched factor + solve of many independent dense systems of uneven order
 * (project addition; the paper factors one matrix).  Systems are grouped into
 * long/short pairs (the pairing idea of Eq. 7 applied across systems: a cheap
 * system joins an expensive one while the pair costs no more than the most
 * expensive system) and run by one persistent kernel launch.
 *
 * ebv_batch_schedule_len(batch): int32 entries of a schedule (2*batch + 8).
 * ebv_batch_schedule (host): builds the schedule for the given orders and
 *   right-hand-side counts (host arrays) into `schedule_host`; EBV_ERR_ARG for
 *   an order outside 0..4096 or a count outside 0..64.  `variant_of_n`
 *   (host, nullable, 4096 entries) maps each order 1..4096 to a kernel
 *   variant id v in 0..EBV_BATCH_VARIANTS-1: block width NB = 16 << (v % 3)
 *   columns and trailing-update output tiles of TM = 64 >> (v / 3) squared
 *   (0: NB 16, TM 64; 1: NB 32, TM 64; 2: NB 64, TM 64; 3..5: the same with
 *   TM 32).  NB = 64 is offered for EBV_FP32 only (in FP64 those ids run as
 *   id 1).  The map usually comes from ebv_batch_autotune; NULL uses the
 *   built-in default (id 0 up to order 64, id 1 above).
 *   The caller copies the schedule to device memory once and may reuse it for
 *   every call with the same sizes.
 * ebv_factor_solve_batched: system s has order n_dev[s] (1..4096) and
 *   nrhs_dev[s] right-hand sides (0..64); a_ptrs_dev[s] points to its n x n
 *   matrix (leading dimension n), overwritten by its packed factors;
 *   b_ptrs_dev[s] to its n x nrhs right-hand sides (leading dimension nrhs),
 *   overwritten by X.  prec is EBV_FP64 or EBV_FP32 (all matrices alike).
 *   info_dev[s] receives the system's pivot status (-1 for an order or count
 *   outside those ranges, found on the device).  ws: workspace of at least
 *   ebv_batch_workspace_size(batch) bytes (a work counter and a status word),
 *   256-byte aligned.  All arrays named _dev are device memory.  Returns
 *   EBV_ERR_ARG for batch outside 0..2^28-1, a precision other than those
 *   two or a null array; EBV_ERR_WORKSPACE for a missing, misaligned or short
 *   ws; EBV_ERR_CUDA when the launch fails (batch 0 returns EBV_OK at once).
 */
EBV_API int64_t ebv_batch_schedule_len(int64_t batch);
EBV_API size_t ebv_batch_workspace_size(int64_t batch);
EBV_API ebv_status_t ebv_batch_schedule(int64_t batch, const int32_t *n_host, const int32_t *nrhs_host,
                                const int8_t *variant_of_n, int32_t *schedule_host);
/*
 * ebv_batch_partition (host): splits a batch across nranks processes, one GPU
 * each, with no exchange between them (the systems are independent; the
 * paper's Abstract and Conclusions name multiple devices as a fit for the
 * method).  The systems are first grouped into the long/short pairs of
 * ebv_batch_schedule (Eq. 7's equalisation across systems); the pairs, in
 * decreasing cost, then go one by one to the rank with the least work so far
 * (lowest rank on ties), so no rank gets more than one pair's cost above the
 * average.  Deterministic: every rank computes the same split from the same
 * sizes.  rank_of_host (host, batch entries) receives each system's rank;
 * cost_of_rank_host (host, nranks entries, nullable) each rank's summed cost
 * in flops (2n^3/3 + 2n^2 nrhs + 1 per system).  EBV_ERR_ARG as for
 * ebv_batch_schedule, or for nranks outside 1..65536.
 */
EBV_API ebv_status_t ebv_batch_partition(int64_t batch, const int32_t *n_host, const int32_t *nrhs_host,
                                         int32_t nranks, int32_t *rank_of_host, double *cost_of_rank_host);
/*
 * ebv_profile_from_band (host): the EBV_PROFILE buffer of a row-band matrix
 * (ab: host, n rows of ldab >= kl+ku+1 doubles, a_ij at ab[i*ldab + j-i+kl]).
 * Each 64-block keeps its part from the first non-zero of its rows / columns
 * outside the diagonal block.  prec EBV_FP64 or EBV_FP32 (the values' type).
 * *bytes_needed receives the buffer size, *kl_out / *ku_out the bounds to
 * pass in the descriptor.  out == NULL only computes those; otherwise out
 * (host, out_bytes >= *bytes_needed, 256-byte aligned for the device copy)
 * receives the buffer, which the caller copies to the device as is.  Any of
 * bytes_needed, kl_out, ku_out may be NULL.  Host only, no device call.
 * EBV_ERR_ARG for n < 1, kl or ku outside 0..n-1, ldab < kl+ku+1 or a null
 * ab; EBV_ERR_UNSUPPORTED for another prec; EBV_ERR_WORKSPACE when out_bytes
 * is short.  (The profile of the sparse matrices of the paper's Table 1,
 * read as uneven bands.)
 */
EBV_API ebv_status_t ebv_profile_from_band(int64_t n, int64_t kl, int64_t ku, const double *ab, int64_t ldab,
                                           ebv_prec_t prec, void *out, size_t out_bytes, size_t *bytes_needed,
                                           int64_t *kl_out, int64_t *ku_out);

EBV_API ebv_status_t ebv_factor_solve_batched(int64_t batch, const int32_t *n_dev, const int32_t *nrhs_dev,
                                      void *const *a_ptrs_dev, void *const *b_ptrs_dev, ebv_prec_t prec,
                                      const int32_t *schedule_dev, int32_t *info_dev, void *ws,
                                      size_t ws_bytes, ebv_stream_t stream);

/*
 * Autotuner for the batched kernel: times every variant offered in `prec` on
 * `reps` synthetic diagonally dominant systems of each order in `orders`
 * (host array of count entries; one launch per variant and order, the
 * second of two runs timed with CUDA events) and writes the fastest variant
 * id per order to best_variant_host.  ms_host (host, nullable, count *
 * EBV_BATCH_VARIANTS entries) receives the times, -1 for variants not
 * offered in `prec`.  scratch_dev must hold ebv_batch_autotune_scratch(max
 * order, reps, prec) bytes, 256-byte aligned.  Synchronises the stream (it
 * measures time).  EBV_ERR_ARG for null orders or best_variant_host, count or
 * reps < 1, an order outside 1..4096 or another precision than EBV_FP64 /
 * EBV_FP32; EBV_ERR_WORKSPACE for a missing, misaligned or short scratch;
 * ebv_batch_autotune_scratch returns 0 for invalid arguments.
 */
#define EBV_BATCH_VARIANTS 6
EBV_API size_t ebv_batch_autotune_scratch(int32_t max_n, int32_t reps, ebv_prec_t prec);
EBV_API ebv_status_t ebv_batch_autotune(const int32_t *orders, int32_t count, int32_t reps, ebv_prec_t prec,
                                void *scratch_dev, size_t scratch_bytes, int8_t *best_variant_host,
                                float *ms_host, ebv_stream_t stream);

/*
 * ebv_inverse -- the explicit inverse from the packed factors, in the product
 * form of Eq. 4c: A^{-1} = U^{-1} L^{-1}, where L^{-1} is the product of the
 * elimination's Gauss transforms and U^{-1} that of the row transforms of U
 * and the pivot scaling.  For many right-hand sides that arrive one by one
 * (X B is one matrix product), not for single solves (ebv_solve is cheaper
 * and more accurate).
 *   desc  dense storage only (band storages: EBV_ERR_UNSUPPORTED);
 *         n and the factors' leading dimension ld.
 *   prec  EBV_FP64 (lu and x binary64) or EBV_FP32 (binary32: the factors of
 *         ebv_factor with EBV_FP32, or the binary32 lowp factors of a
 *         mixed-precision factorisation); others give EBV_ERR_UNSUPPORTED.
 *   lu    device, the packed factors (L strictly below the diagonal, unit
 *         diagonal implied; U on and above), row-major; read only.  They must
 *         come from a factorisation whose info was 0: zero pivots are not
 *         checked here and give non-finite entries in x.
 *   x     device output, n x n, row-major, leading dimension ldx >= n; it
 *         must not overlap lu (EBV_ERR_ARG) and serves as scratch until the
 *         last launch writes A^{-1}.
 *   ws    device workspace, 256-byte aligned, of at least
 *         ebv_inverse_workspace_size(n, prec) bytes (the packed inverses of the
 *         two triangles: n x n elements); EBV_ERR_WORKSPACE otherwise.
 * Work: 4n^3/3 flops in 2 + 2*ceil(log2(n/64)) launches on `stream`; no host
 * synchronisation, capturable.  n <= 2^21.
 */
EBV_API size_t ebv_inverse_workspace_size(int64_t n, ebv_prec_t prec);
EBV_API ebv_status_t ebv_inverse(const ebv_desc_t *desc, ebv_prec_t prec, const void *lu, void *x, int64_t ldx,
                                 void *ws, size_t ws_bytes, ebv_stream_t stream);

/*
 * ebv_solve_adjoint -- gradients of X = A^{-1} B for a batch of equal-size
 * FP64 systems (project addition; the paper has no gradients).  From the
 * stored factors (A = LU, so A^T = U^T L^T):
 *   grad_B = A^{-T} grad_X   (U^T z = grad_X forward, then L^T w = z backward),
 *   grad_A = -grad_B X^T.
 *   lu        device, system s at lu + s*stride_lu, leading dimension lda.
 *   x, grad_x device, system s at + s*n*nrhs (n x nrhs, leading dim. nrhs).
 *   grad_b    device output, same layout as x.
 *   grad_a    device output or NULL, system s at + s*n*n (leading dim. n).
 * Limits: batch <= 65535, nrhs <= 16, and with grad_a one system's X (n*nrhs
 * doubles) must fit in 200 KB of shared memory (EBV_ERR_UNSUPPORTED otherwise).
 */
EBV_API ebv_status_t ebv_solve_adjoint(int64_t batch, int64_t n, int64_t nrhs, const double *lu, int64_t lda,
                               int64_t stride_lu, const double *x, const double *grad_x, double *grad_b,
                               double *grad_a, ebv_stream_t stream);

/*
 * ebv_gesv_host -- X = A^{-1} B for A and B in HOST memory (Eq. 1 with the
 * factorisation of Eq. 6-7 and refinement), mixed precisions only
 * (EBV_MIXED_BF16 / EBV_MIXED_FP16), dense storage.  The host-to-device copy
 * of A runs on an internal stream, column block by column block, and the
 * factorisation starts on the first block while the rest is still in
 * flight (the recursion reaches the columns of A from left to right); then B
 * is solved and refined exactly as by ebv_factor + ebv_solve, and X is
 * copied back to x_host.  Everything is ordered on `stream`: the results
 * (x_host, *report_host, *info_host) are valid once the stream has
 * completed.  Host buffers should be page-locked for the copies to overlap.
 *
 *   a_host      host double*, n x n, leading dimension desc->ld (not modified).
 *   b_host      host double*, n x nrhs, leading dimension ldb (not modified).
 *   x_host      host double*, n x nrhs, leading dimension ldb: receives X (may be b_host).
 *   refine      as for ebv_solve (NULL: the unrefined mixed-precision solve).
 *   report_host host ebv_refine_report_t (written when refine != NULL; may be NULL).
 *   info_host   host int32 (may be NULL): 0 or the first bad pivot, as for ebv_factor.
 *   ws          device workspace of ebv_gesv_host_workspace_size(desc, prec,
 *               nrhs) bytes, 256-byte aligned: the device copies of A (FP64),
 *               of the factors (FP32) and of B / X, and the factor / solve
 *               workspaces.
 * The first call on a device creates the internal stream and events (make it
 * before any stream capture); later calls reuse them, so calls on one device
 * must be ordered (e.g. one stream).  EBV_ERR_UNSUPPORTED for other
 * precisions or band storage.
 */
EBV_API size_t ebv_gesv_host_workspace_size(const ebv_desc_t *desc, ebv_prec_t prec, int64_t nrhs);
EBV_API ebv_status_t ebv_gesv_host(const ebv_desc_t *desc, ebv_prec_t prec, const double *a_host,
                                   const double *b_host, double *x_host, int64_t nrhs, int64_t ldb,
                                   const ebv_refine_t *refine,
                                   ebv_refine_report_t *report_host, int32_t *info_host, void *ws, size_t ws_bytes,
                                   ebv_stream_t stream);

/*
 * ebv_solve_static -- ebv_solve without a caller-supplied workspace, for
 * callers that cannot allocate device memory (code running while someone
 * else captures the stream into a CUDA graph, loops whose memory is budgeted
 * up front, plug-ins whose host owns every allocation).  The paper has no
 * counterpart: it is an interface addition of this library.
 *
 * Arguments, layouts, ownership and results are those of ebv_solve; the
 * workspace is a fixed device array of EBV_STATIC_SCRATCH_BYTES inside this
 * library, reserved on every device that loads it until the process exits.
 * The call allocates nothing (no cudaMalloc, cudaFree or allocating library
 * routine).
 *
 * Limits: n <= EBV_STATIC_MAX_N and nrhs <= EBV_STATIC_MAX_NRHS; larger
 * sizes return EBV_ERR_WORKSPACE before any work is enqueued.
 *
 * The first call in a CUDA context looks up the array's device address
 * (cudaGetSymbolAddress) with that context current; make that first call
 * before any stream capture in it.  The address is cached per device with
 * the context's unique ID and looked up again when another context is
 * current: after cudaDeviceReset (which makes a new primary context) or when
 * the caller has made a context of its own current, the next call is such a
 * first call again.  All calls on a device share the one array, which keeps
 * the last call's contents (each call clears what has to start at zero):
 * calls whose work overlaps on the GPU (other streams, other host threads
 * without ordering) race and give undefined results.
 */
#define EBV_STATIC_SCRATCH_BYTES ((size_t)20 << 20)
#define EBV_STATIC_MAX_N 4096
#define EBV_STATIC_MAX_NRHS 32
EBV_API ebv_status_t ebv_solve_static(const ebv_desc_t *desc, ebv_prec_t prec, const void *lu,
                                      const double *a_orig, void *b, int64_t nrhs, int64_t ldb,
                                      const ebv_refine_t *refine, ebv_refine_report_t *report_dev,
                                      ebv_stream_t stream);

/*
 * Testing hook (no counterpart in the paper): selects how the mixed-precision
 * trailing updates run.  0 = automatic (tensor cores where the shape allows),
 * 1 = SIMT FP32 kernel from the same bfloat16/half operands, 2 = tensor cores
 * only.  Process-wide; not for concurrent use with running factorisations.
 */
EBV_API void ebv_debug_set_lowp_gemm(int32_t mode);

/*
 * Testing hooks of the thread-block-cluster panel kernel, which factors a
 * panel (its diagonal block, L21 and U12) in one launch on up to 16 CTAs,
 * the panel's columns paired long with short over the CTAs (Eq. 7), the
 * pivot column passed through distributed shared memory (or L2 for tall
 * panels).  ebv_debug_set_band_cluster(1) makes the banded factorisation use
 * it for every 64-column panel (default 0: the diagonal block on one CTA and
 * L21 / U12 as separate launches, measured faster).  ebv_debug_set_cluster_panel
 * (0) switches the kernel off wherever it would run (default 1).  The
 * results agree to rounding.  Process-wide.
 */
EBV_API void ebv_debug_set_band_cluster(int32_t enable);
/* Testing hook: the FP64 band panels' overlaps on internal side streams.
 * 0 = all serial; 1 = the symmetric storages' look-ahead (the next panel's
 * diagonal block under the rest of the trailing update) and, for the general
 * band, each panel's U12 beside its L21; 2 (default) = also the look-ahead for
 * the general band.  The same results in every mode.  Process-wide. */
EBV_API void ebv_debug_set_band_lookahead(int32_t mode);
EBV_API void ebv_debug_set_cluster_panel(int32_t enable);
/* Testing hook: 0 = the FP64 panels' 64 x 64 diagonal blocks (band storages,
 * dense FP64 systems of order <= 256) on the blocked 16 x 16 sub-block
 * kernel instead of the register-resident one (default 1).  Both compute
 * the same Doolittle factors; the rounding of the updates may differ.
 * Process-wide. */
EBV_API void ebv_debug_set_diag_lu(int32_t enable);

/*
 * Testing hook: dense FP64 systems of order <= 256 are factored as
 * right-looking 64-column panels (the diagonal block on one CTA without its
 * inverses, L21 and U12 by substitution on many CTAs, one trailing update)
 * and solved by one CTA's block substitution when panels != 0 (default);
 * else factored on one thread-block cluster and solved by the general
 * substitution kernels.  The results agree to rounding.  Process-wide.
 */
EBV_API void ebv_debug_set_small_dense(int32_t panels);

/*
 * Testing hook: the banded factorisation (every band storage) first finds
 * the block envelope of A -- per 64-block, the first non-zero left of the
 * diagonal over the block's rows and above it over its columns -- and skips
 * the L21, U12 and trailing-update tiles that lie outside it (no row exchanges,
 * so the factors never leave the envelope; a band whose width varies row by
 * row costs the work of its profile).  enable = 0 switches the skipping off;
 * the factors are the same bit for bit.  Process-wide, default on.
 */
EBV_API void ebv_debug_set_band_envelope(int32_t enable);

/*
 * Testing hook (project addition; the aggregated rank-1 update of Eq. 6c as
 * the mixed-precision factorisation runs it):
 *   C(m0+i, n0+j) -= scale[2] * sum_{k<K} lb(m0+i, k0+k) * ut(n0+j, k0+k)
 * for 0 <= i < M, 0 <= j < N.  op: 0 = bfloat16 operands, 1 = half.  engine:
 * 1 = SIMT FP32 kernel, 2 = tcgen05 tensor-core kernel (returns
 * EBV_ERR_UNSUPPORTED unless K is a multiple of 64, k0 of 8, ldsh*2 of 16 and
 * lb, ut are 16-byte aligned).  C: device float, row stride ldc.  lb, ut:
 * device 16-bit matrices with row stride ldsh.  scale: device float[3].
 * ws: 256-byte-aligned device scratch of at least 256 bytes (status block).
 */
EBV_API ebv_status_t ebv_debug_lowp_update(int32_t op, int32_t engine, float *C, int64_t ldc, const void *lb,
                                           const void *ut, int64_t ldsh, const float *scale, int64_t m0, int64_t n0,
                                           int64_t k0, int64_t M, int64_t N, int64_t K, void *ws,
                                           ebv_stream_t stream);
/* 1 when the tensor-map encoder of the CUDA driver could be resolved. */
EBV_API int32_t ebv_debug_tc_available(void);

/*
 * Failure-detection probe (project addition): runs the library's bounded
 * device wait for `polls` polls (1 .. 2^22) on a flag in `ws` that nothing
 * sets.  Afterwards the status block at the start of ws (int32 code, where,
 * done, pad) reads EBV_ERR_TIMEOUT, 77, 0, 1: the wait expired, the status was
 * recorded and the kernel went on and returned.  ws: >= 256 bytes, 256-aligned.
 */
EBV_API ebv_status_t ebv_debug_wait_probe(int64_t polls, void *ws, ebv_stream_t stream);

/*
 * Testing hook (project addition; the residual of the refinement loop):
 * R = B - A X for a dense FP64 A (n x n, lda) and FP64 X, B (n x nrhs,
 * leading dimension nrhs), evaluated exactly as ebv_solve's dense refinement
 * does it: on the tensor cores by exact splitting of A and X into integer
 * digits (products and partial sums exact in the FP32 accumulators, the
 * digit-pair sums carried in triple-binary32), accurate to FP64 level;
 * without the tensor-map encoder, the triple-binary32 SIMT kernel.
 * R: device, n x nrhs.  ws: a workspace of at least
 * ebv_workspace_size(dense n, EBV_FP64, nrhs) bytes.
 */
EBV_API ebv_status_t ebv_debug_residual(int64_t n, const double *a, int64_t lda, const double *x, const double *b,
                                        int64_t nrhs, double *r, void *ws, size_t ws_bytes, ebv_stream_t stream);

/*
 * Instrumentation (no counterpart in the paper).
 * ebv_debug_launch_count: kernels launched by this library so far (process-wide).
 * ebv_debug_profile(1) brackets every later launch with CUDA events on its
 * stream, per kernel class: 0 mixed-precision trailing update, 1 working-
 * precision trailing update, 2 diagonal blocks, 3 block substitutions,
 * 4 refinement residual, 5 batched kernel, 6 adjoint, 7 other, 8 U12
 * tile products and blocked TRSMs, 9 L21 tile products, 10 two-leaf middle
 * step (U12 and the trailing update of a 128-column node in one launch),
 * 11 explicit inverse (ebv_inverse).
 * ebv_debug_profile_read fills, for the 12 classes, the summed device time in
 * ms, the summed algorithmic work (flops) and the launch count of the launches
 * recorded since the previous read (host arrays of 12; synchronises on the
 * recorded events).  Profiling adds an event pair per launch; switch it off
 * for timed runs.
 */
EBV_API int64_t ebv_debug_launch_count(void);
EBV_API void ebv_debug_profile(int32_t enable);
EBV_API int32_t ebv_debug_profile_read(double *ms_by_class, double *work_by_class, int64_t *count_by_class);

#ifdef __cplusplus
}
#endif

#endif /* EBV_H_ */
