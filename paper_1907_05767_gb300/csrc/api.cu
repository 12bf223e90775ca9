// C ABI of the EbV library: argument checks and dispatch.  Every check runs
// on the host before anything is enqueued, so invalid calls return EBV_ERR_ARG
// without touching the GPU.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

using namespace ebv;

namespace {

constexpr int64_t kMaxN = int64_t(1) << 30;
// Largest order of the explicit inverse (its level launches put two nodes per
// grid.z slot, its product one CTA per tile in grid.x).
constexpr int64_t kMaxInverseN = int64_t(1) << 21;

// Runs the library's bounded wait on flag (which the caller leaves at 0, so
// nothing ever sets it): every thread of the CTA returns after `polls` polls
// and the status block records EBV_ERR_TIMEOUT.
__global__ void k_probe_wait(const int *flag, DevStatus *st, long long polls) {
  __shared__ int ok;
  if (threadIdx.x == 0) ok = bounded_wait_geq(flag, 1, st, polls, 77);
  __syncthreads();
  if (!ok && threadIdx.x == 0) st->pad = 1;  // the CTA went on after the expired wait
}

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

size_t elem_size(ebv_prec_t p) { return p == EBV_FP32 ? 4 : 8; }

bool valid_prec(ebv_prec_t p) {
  return p == EBV_FP64 || p == EBV_FP32 || p == EBV_MIXED_BF16 || p == EBV_MIXED_FP16;
}
bool is_mixed(ebv_prec_t p) { return p == EBV_MIXED_BF16 || p == EBV_MIXED_FP16; }

ebv_status_t check_desc(const ebv_desc_t *d, ebv_prec_t prec) {
  if (!d || !valid_prec(prec)) return EBV_ERR_ARG;
  if (d->n < 0 || d->n > kMaxN) return EBV_ERR_ARG;
  if (d->storage == EBV_DENSE || d->storage == EBV_DENSE_SYM) {
    if (d->ld < std::max<int64_t>(1, d->n)) return EBV_ERR_ARG;
  } else if (d->storage == EBV_BAND || d->storage == EBV_BAND_SYM || d->storage == EBV_BAND_SYM_LOWER) {
    if (d->kl < 0 || d->ku < 0) return EBV_ERR_ARG;
    if (d->storage != EBV_BAND && d->kl != d->ku) return EBV_ERR_ARG;
    if (d->n > 0 && (d->kl >= d->n || d->ku >= d->n)) return EBV_ERR_ARG;
    if (d->ld < (d->storage == EBV_BAND_SYM_LOWER ? d->kl + 1 : d->kl + d->ku + 1)) return EBV_ERR_ARG;
  } else if (d->storage == EBV_PROFILE) {
    if (d->kl < 0 || d->ku < 0) return EBV_ERR_ARG;
    if (d->n > 0 && (d->kl >= d->n || d->ku >= d->n)) return EBV_ERR_ARG;
  } else {
    return EBV_ERR_ARG;
  }
  return EBV_OK;
}

}  // namespace

extern "C" {

int32_t ebv_version(void) { return 100; }

const char *ebv_status_string(ebv_status_t s) {
  switch (s) {
    case EBV_OK: return "ok";
    case EBV_ERR_ARG: return "invalid argument";
    case EBV_ERR_ZERO_PIVOT: return "zero pivot";
    case EBV_ERR_NONFINITE: return "non-finite pivot";
    case EBV_ERR_NOT_CONVERGED: return "refinement did not converge";
    case EBV_ERR_TIMEOUT: return "device wait timed out";
    case EBV_ERR_CUDA: return "CUDA error";
    case EBV_ERR_UNSUPPORTED: return "unsupported combination";
    case EBV_ERR_WORKSPACE: return "workspace missing or too small";
  }
  return "unknown status";
}

size_t ebv_workspace_size(const ebv_desc_t *desc, ebv_prec_t prec, int64_t nrhs) {
  if (check_desc(desc, prec) != EBV_OK || nrhs < 0) return 0;
  const int64_t n = desc->n;
  if (desc->storage != EBV_DENSE)
    return std::max(band_factor_ws(n, ws_kl(desc), desc->ku, prec), band_solve_ws(n, nrhs, prec));
  return std::max(dense_factor_ws(n, prec), dense_solve_ws(n, nrhs, prec));
}

ebv_status_t ebv_factor(const ebv_desc_t *desc, ebv_prec_t prec, void *a, void *lowp, int32_t *info_dev, void *ws,
                        size_t ws_bytes, ebv_stream_t stream) {
  EBV_TRY(check_desc(desc, prec));
  if (!info_dev || !aligned(info_dev, 4)) return EBV_ERR_ARG;
  if (desc->n > 0 && (!a || !aligned(a, desc->storage == EBV_PROFILE ? 256 : elem_size(prec)))) return EBV_ERR_ARG;
  if ((desc->storage == EBV_PROFILE || desc->storage == EBV_DENSE_SYM) && is_mixed(prec)) return EBV_ERR_UNSUPPORTED;
  if (is_mixed(prec) && desc->n > 0 && (!lowp || !aligned(lowp, 16))) return EBV_ERR_ARG;
  if (ws && !aligned(ws, 256)) return EBV_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (desc->storage != EBV_DENSE) {
    if (!ws || ws_bytes < band_factor_ws(desc->n, ws_kl(desc), desc->ku, prec)) return EBV_ERR_WORKSPACE;
    return band_factor(desc, prec, a, lowp, info_dev, ws, ws_bytes, s);
  }
  const size_t need = dense_factor_ws(desc->n, prec);
  if (need > 0 && (!ws || ws_bytes < need)) return EBV_ERR_WORKSPACE;
  return dense_factor(desc, prec, a, lowp, info_dev, ws, ws_bytes, s);
}

ebv_status_t ebv_solve(const ebv_desc_t *desc, ebv_prec_t prec, const void *lu, const double *a_orig, void *b,
                       int64_t nrhs, int64_t ldb, const ebv_refine_t *refine, ebv_refine_report_t *report_dev,
                       void *ws, size_t ws_bytes, ebv_stream_t stream) {
  EBV_TRY(check_desc(desc, prec));
  if (nrhs < 0 || nrhs > (int64_t(1) << 20) || ldb < std::max<int64_t>(1, nrhs)) return EBV_ERR_ARG;
  const bool any = desc->n > 0 && nrhs > 0;
  const size_t bsz = prec == EBV_FP32 ? 4 : 8;
  const size_t fsz = prec == EBV_FP64 ? 8 : 4;
  if (any && (!lu || !aligned(lu, desc->storage == EBV_PROFILE ? 256 : fsz) || !b || !aligned(b, bsz))) return EBV_ERR_ARG;
  if ((desc->storage == EBV_PROFILE || desc->storage == EBV_DENSE_SYM) && is_mixed(prec)) return EBV_ERR_UNSUPPORTED;
  const bool need_a = is_mixed(prec) && refine;
  if (refine) {
    if (!(refine->tol >= 0.0) || refine->max_iter < 0 || refine->max_iter > 1000) return EBV_ERR_ARG;
    if (prec == EBV_FP32) return EBV_ERR_UNSUPPORTED;  // refinement returns FP64 solutions
  }
  if ((need_a || refine) && any && (!a_orig || !aligned(a_orig, 8))) return EBV_ERR_ARG;
  if (report_dev && !aligned(report_dev, 8)) return EBV_ERR_ARG;
  if (!ws || !aligned(ws, 256)) return EBV_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  if (desc->storage != EBV_DENSE)
    return band_solve(desc, prec, lu, a_orig, b, nrhs, ldb, refine, report_dev, ws, ws_bytes, s);
  return dense_solve(desc, prec, lu, a_orig, b, nrhs, ldb, refine, report_dev, ws, ws_bytes, s);
}

size_t ebv_inverse_workspace_size(int64_t n, ebv_prec_t prec) {
  if (n < 0 || n > kMaxInverseN || (prec != EBV_FP64 && prec != EBV_FP32)) return 0;
  return inverse_ws(n, prec);
}

ebv_status_t ebv_inverse(const ebv_desc_t *desc, ebv_prec_t prec, const void *lu, void *x, int64_t ldx, void *ws,
                         size_t ws_bytes, ebv_stream_t stream) {
  EBV_TRY(check_desc(desc, prec));
  if (desc->storage != EBV_DENSE || (prec != EBV_FP64 && prec != EBV_FP32)) return EBV_ERR_UNSUPPORTED;
  const int64_t n = desc->n;
  if (n > kMaxInverseN) return EBV_ERR_UNSUPPORTED;
  if (ldx < std::max<int64_t>(1, n)) return EBV_ERR_ARG;
  if (n == 0) return EBV_OK;
  const size_t es = elem_size(prec);
  if (!lu || !x || !aligned(lu, es) || !aligned(x, es)) return EBV_ERR_ARG;
  const uintptr_t l0 = (uintptr_t)lu, l1 = l0 + ((n - 1) * desc->ld + n) * es;
  const uintptr_t x0 = (uintptr_t)x, x1 = x0 + ((n - 1) * ldx + n) * es;
  if (l0 < x1 && x0 < l1) return EBV_ERR_ARG;  // X is written while the factors are still read
  if (!ws || !aligned(ws, 256) || ws_bytes < inverse_ws(n, prec)) return EBV_ERR_WORKSPACE;
  return inverse(n, prec, lu, desc->ld, x, ldx, ws, (cudaStream_t)stream);
}

// Testing hook: 0 = small dense FP64 systems on one thread-block cluster
// instead of substitution panels.
void ebv_debug_set_small_dense(int32_t panels) { set_small_dense_panels(panels != 0); }

// Testing hook: 0 = FP64 panels' diagonal blocks on the blocked sub-block kernel.
void ebv_debug_set_diag_lu(int32_t enable) { set_diag_lu(enable != 0); }

// Testing hook: FP64 band panels' overlaps, 0 = serial, 1 = default, 2 = also
// the general band's look-ahead.
void ebv_debug_set_band_lookahead(int32_t mode) { set_band_overlap(mode < 0 ? 0 : mode > 2 ? 2 : mode); }

// Testing hook: 1 = band panels on thread-block clusters.
void ebv_debug_set_band_cluster(int32_t enable) { set_band_cluster(enable != 0); }

// Testing hook: 0 = panels never run on a thread-block cluster.
void ebv_debug_set_cluster_panel(int32_t enable) { set_cluster_panel(enable != 0); }

// Testing hook: 0 = the banded factorisation ignores the block envelope.
void ebv_debug_set_band_envelope(int32_t enable) { set_band_envelope(enable != 0); }

// Testing hook: 0 = automatic, 1 = SIMT only, 2 = tensor cores where possible.
void ebv_debug_set_lowp_gemm(int32_t mode) { set_lowp_gemm_mode(mode); }

ebv_status_t ebv_debug_lowp_update(int32_t op, int32_t engine, float *C, int64_t ldc, const void *lb, const void *ut,
                                   int64_t ldsh, const float *scale, int64_t m0, int64_t n0, int64_t k0, int64_t M,
                                   int64_t N, int64_t K, void *ws, ebv_stream_t stream) {
  if ((op != 0 && op != 1) || (engine != 1 && engine != 2)) return EBV_ERR_ARG;
  if (M < 0 || N < 0 || K < 0 || m0 < 0 || n0 < 0 || k0 < 0 || ldsh < k0 + K || ldc < n0 + N) return EBV_ERR_ARG;
  if (M == 0 || N == 0 || K == 0) return EBV_OK;
  if (!C || !lb || !ut || !scale || !ws || !aligned(ws, 256)) return EBV_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(ws, 0, sizeof(DevStatus), s) != cudaSuccess) return EBV_ERR_CUDA;
  if (engine == 2)
    return tc_update(op, C, ldc, lb, ut, ldsh, scale, m0, n0, k0, M, N, K, (DevStatus *)ws, s);
  return simt_update(op, C, ldc, lb, ut, ldsh, scale, m0, n0, k0, M, N, K, s);
}

int32_t ebv_debug_tc_available(void) { return tc_available() ? 1 : 0; }

ebv_status_t ebv_debug_wait_probe(int64_t polls, void *ws, ebv_stream_t stream) {
  if (polls < 1 || polls > kSpinLimit) return EBV_ERR_ARG;
  if (!ws || ((uintptr_t)ws % 256) != 0) return EBV_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  EBV_CU(cudaMemsetAsync(ws, 0, kStatusBytes, s));  // status block and the flag at byte 64
  k_probe_wait<<<1, 64, 0, s>>>((const int *)((char *)ws + 64), (DevStatus *)ws, polls);
  return launch_ok();
}

ebv_status_t ebv_debug_residual(int64_t n, const double *a, int64_t lda, const double *x, const double *b,
                                int64_t nrhs, double *r, void *ws, size_t ws_bytes, ebv_stream_t stream) {
  if (n < 0 || nrhs < 0 || lda < std::max<int64_t>(1, n)) return EBV_ERR_ARG;
  if (n == 0 || nrhs == 0) return EBV_OK;
  if (!a || !x || !b || !r || !aligned(a, 8) || !aligned(x, 8) || !aligned(b, 8) || !aligned(r, 8)) return EBV_ERR_ARG;
  if (!ws || !aligned(ws, 256)) return EBV_ERR_WORKSPACE;
  return debug_residual(n, a, lda, x, b, nrhs, r, ws, ws_bytes, (cudaStream_t)stream);
}

}  // extern "C"
