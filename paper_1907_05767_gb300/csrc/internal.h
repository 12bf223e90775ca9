// Internal interfaces between the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "ebv.h"

namespace ebv {

// Workspace bytes of the dense paths.
size_t dense_factor_ws(int64_t n, ebv_prec_t prec);
size_t dense_solve_ws(int64_t n, int64_t nrhs, ebv_prec_t prec);
size_t band_factor_ws(int64_t n, int64_t kl, int64_t ku, ebv_prec_t prec);
// The lower band width that sizes the band paths' workspace (the dense
// symmetric storage ignores desc->kl and never runs the cluster panels).
inline int64_t ws_kl(const ebv_desc_t *d) { return d->storage == EBV_DENSE_SYM ? 0 : d->kl; }
size_t band_solve_ws(int64_t n, int64_t nrhs, ebv_prec_t prec);

ebv_status_t dense_factor(const ebv_desc_t *d, ebv_prec_t prec, void *a, void *lowp, int32_t *info, void *ws,
                          size_t ws_bytes, cudaStream_t s);
ebv_status_t dense_solve(const ebv_desc_t *d, ebv_prec_t prec, const void *lu, const double *a_orig, void *b,
                         int64_t nrhs, int64_t ldb, const ebv_refine_t *refine, ebv_refine_report_t *rep, void *ws,
                         size_t ws_bytes, cudaStream_t s);
unsigned int *dense_factor_scan_init(int64_t n, ebv_prec_t prec, void *ws, cudaStream_t s);
ebv_status_t dense_factor_staged(int64_t n, ebv_prec_t prec, const double *a_dev, float *lowp, int32_t *info,
                                 void *ws, size_t ws_bytes, const cudaEvent_t *ev, int64_t cbw, bool convert,
                                 cudaStream_t s);
ebv_status_t band_factor(const ebv_desc_t *d, ebv_prec_t prec, void *a, void *lowp, int32_t *info, void *ws,
                         size_t ws_bytes, cudaStream_t s);
// Testing hook of the banded factorisation: false = no block envelope (every
// CTA of the band window works; the results are the same).
void set_band_envelope(bool on);
// Testing hook: true = band panels on thread-block clusters (default false).
void set_band_cluster(bool on);
// Testing hook: false = FP64 band panels without look-ahead (default true).
void set_band_overlap(int mode);
void set_diag_lu(bool on);
// Dense FP64 factorisation of a small system as right-looking 64-column
// panels (band.cu); orders up to kSmallDenseMaxN use it.
ebv_status_t dense_small_factor(double *a, int64_t ld, int64_t n, int32_t *info, void *ws, cudaStream_t s);
constexpr int64_t kSmallDenseMaxN = 256;
void set_small_dense_panels(bool on);
ebv_status_t band_solve(const ebv_desc_t *d, ebv_prec_t prec, const void *lu, const double *a_orig, void *b,
                        int64_t nrhs, int64_t ldb, const ebv_refine_t *refine, ebv_refine_report_t *rep, void *ws,
                        size_t ws_bytes, cudaStream_t s);

// Panel factorisation on a thread-block cluster (cluster_panel.cu): the W
// columns [c0, c0+W) of rows [c0, c0+R) factored (packed L\U of the diagonal
// block and L21), and U12 = L11^{-1} A12 formed in place for the U columns
// right of the panel, on the view base[i*ld + j] (zero outside -kl..ku).
// EBV_ERR_UNSUPPORTED when the shape does not fit the kernel or the device
// cannot run the cluster (the caller then uses the one-CTA leaf kernels).
// symlo: only the lower half of a symmetric band is stored (U must be 0).
// bcast: device scratch of 2 (R + 1) elements (or null) through which tall
// panels pass the pivot column in L2 instead of distributed shared memory.
bool cluster_panel_fits(bool fp64, int W, int64_t R, int64_t U);
ebv_status_t cluster_panel(bool fp64, void *base, int64_t ld, int64_t kl, int64_t ku, bool symlo, int64_t c0, int W,
                           int64_t R, int64_t U, int32_t *info, void *bcast, cudaStream_t s);
// Testing hook: false = never use the cluster panel kernel.
void set_cluster_panel(bool on);
bool cluster_panel_enabled();
// Orders up to which a dense FP64 / FP32 factorisation is one cluster panel.
constexpr int64_t kClusterDenseMaxN = 256;

// Product-form inverse (Eq. 4c) from packed dense factors (inverse.cu).
size_t inverse_ws(int64_t n, ebv_prec_t prec);
ebv_status_t inverse(int64_t n, ebv_prec_t prec, const void *lu, int64_t ldl, void *x, int64_t ldx, void *ws,
                     cudaStream_t s);

struct DevStatus;

// Mixed-precision trailing update C(m0.., n0..) -= scale[2] * lb(m0.., k0..) * ut(n0.., k0..)^T
// (op 0 = bfloat16 operands, 1 = half).  Uses the tcgen05 kernel when the
// shape allows it, else the SIMT kernel.  st: device status block (timeouts).
ebv_status_t lowp_update(int op, float *C, int64_t ldc, const void *lb, const void *ut, int64_t ldsh,
                         const float *scale, int64_t m0, int64_t n0, int64_t k0, int64_t M, int64_t N, int64_t K,
                         DevStatus *st, cudaStream_t s);

// tcgen05 GEMM (tc_gemm.cu).  Returns EBV_ERR_UNSUPPORTED when the shape or
// alignment does not fit the kernel (the caller then uses the SIMT kernel).
ebv_status_t tc_update(int op, float *C, int64_t ldc, const void *lb, const void *ut, int64_t ldsh,
                       const float *scale, int64_t m0, int64_t n0, int64_t k0, int64_t M, int64_t N, int64_t K,
                       DevStatus *st, cudaStream_t s);
bool tc_available();
// 2-D tensor map of a bfloat16 matrix (cols contiguous, row stride ld_elems)
// with the given box and swizzle (128, 64, 32 or 0 bytes).
bool make_map_bf16(CUtensorMap *map, const void *base, int64_t cols, int64_t rows, int64_t ld_elems, int box_cols,
                   int box_rows, int swizzle_bytes);

// FP64-accurate R = B - A X on the tensor cores (exact digit splitting).
// ws: residual_tc_ws(n, nrhs) bytes; rows_ready: the per-row exponents of A
// are already in ws from an earlier call with the same A.
size_t residual_tc_ws(int64_t n, int64_t nrhs);
ebv_status_t residual_tc(const double *A, int64_t lda, int64_t n, const double *X, int64_t ldx, int64_t nrhs,
                         const double *B, int64_t ldb, double *R, int64_t ldr, unsigned long long *rmax, void *ws,
                         bool rows_ready, DevStatus *st, cudaStream_t s);
ebv_status_t simt_update(int op, float *C, int64_t ldc, const void *lb, const void *ut, int64_t ldsh,
                         const float *scale, int64_t m0, int64_t n0, int64_t k0, int64_t M, int64_t N, int64_t K,
                         cudaStream_t s);

// 0 = automatic, 1 = force SIMT, 2 = force tensor cores (testing hooks).
void set_lowp_gemm_mode(int mode);
int get_lowp_gemm_mode();

}  // namespace ebv

namespace ebv {
ebv_status_t debug_residual(int64_t n, const double *a, int64_t lda, const double *x, const double *b, int64_t nrhs,
                            double *r, void *ws, size_t ws_bytes, cudaStream_t s);
}  // namespace ebv
