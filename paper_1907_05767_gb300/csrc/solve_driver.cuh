// Solve orchestration shared by the dense and banded paths: block substitutions
// (Eq. 1) and iterative refinement with an FP64-accurate residual.
#pragma once

#include <algorithm>

#include "solve_kernels.cuh"

namespace ebv {
namespace {

// Right-hand sides per substitution chain (RC): each chunk of RC columns is
// solved by its own chain of CTAs.  One chain of 32 reads the factors once
// and, up to n = 64 x (resident CTAs), gives every CTA a single row block,
// so no CTA has a backlog of folds when its block's turn comes.  Up to 8
// right-hand sides take chunks of 8 instead: the products cover whole
// chunks, and 32-wide ones would spend 3/4 of the arithmetic on zero columns.
// NS: stages of the factor-tile ring; MINB: CTAs per SM the kernel is
// compiled for.
template <typename T, int RCW = 32>
struct TrsvCfg {
  static constexpr int RC = RCW;
  static constexpr int NS = sizeof(T) == 4 ? 3 : 2;
  static constexpr int MINB = RCW == 32 ? (sizeof(T) == 4 ? 2 : 1) : (sizeof(T) == 4 ? 3 : 2);
};

struct DenseSolveLayout {
  size_t dinv, xw, bsave, r, corr, xhi, xlo, rmax, bmax, tcres, total;
};

// Solve workspace: status block, inverses of the diagonal blocks of both
// factors, the substitutions' published blocks, refinement buffers (and,
// for the dense path, the tensor-core residual's exponents and digit planes).
DenseSolveLayout solve_layout(int64_t n, int64_t nrhs, size_t tsize, bool tc_residual = false) {
  DenseSolveLayout L{};
  size_t off = kStatusBytes;
  const size_t nn = (size_t)n * (size_t)std::max<int64_t>(nrhs, 1);
  const size_t nblk = (size_t)std::max<int64_t>(1, (n + kNB - 1) / kNB);
  const size_t rcols = (size_t)std::max<int64_t>(1, (nrhs + 31) / 32) * 32;  // nrhs rounded up to chunks of 32
  L.dinv = off; off = align256(off + nblk * 4 * kNB * kNB * tsize);
  // published solution blocks of the substitutions (tagged words; both triangles use it in turn)
  L.xw = off; off = align256(off + rcols * nblk * kNB * (tsize / 4) * sizeof(unsigned long long));
  L.bsave = off; off = align256(off + nn * 8);
  L.r = off; off = align256(off + nn * 8);
  L.corr = off; off = align256(off + nn * tsize);
  L.xhi = off; off = align256(off + nn * 4);
  L.xlo = off; off = align256(off + nn * 4);
  L.rmax = off; off = align256(off + (size_t)std::max<int64_t>(nrhs, 1) * 8);
  L.bmax = off; off = align256(off + (size_t)std::max<int64_t>(nrhs, 1) * 8);
  L.tcres = off; off = align256(off + (tc_residual ? residual_tc_ws(n, std::max<int64_t>(nrhs, 1)) : 0));
  L.total = off;
  return L;
}

inline int grid_for(int64_t elems) { return (int)std::min<int64_t>(4096, std::max<int64_t>(1, (elems + 255) / 256)); }

// Inverses of the diagonal blocks of the factors (once per solve call).
template <typename T, bool XV>
ebv_status_t diag_inverses(MatView<T, XV> F, int64_t n, T *dinv, cudaStream_t s) {
  static const cudaError_t attr = set_smem(k_diag_inverses<T, kNB, XV>, (int)diag_smem_bytes<T, kNB>());
  if (attr != cudaSuccess) return EBV_ERR_CUDA;
  prof::Scope ps(s, prof::kTrsv, 2.0 * ceil_div(n, kNB) * kNB * kNB * kNB * (2.0 / 3.0 + 4.0));
  k_diag_inverses<T, kNB><<<ceil_div(n, kNB), 4 * kNB, diag_smem_bytes<T, kNB>(), s>>>(F, n, dinv);
  return launch_ok();
}

// One triangle of the substitution as a cooperative persistent launch: at
// most as many CTAs per right-hand-side chunk as can be resident at once
// (the CTAs wait on one another's published blocks).
template <typename T, bool UPPER, int RCW, bool XV>
ebv_status_t trsv_launch(MatView<T, XV> F, int64_t n, T *B, int64_t ldb, int nrhs, const T *dinv,
                         unsigned long long *xw, DevStatus *st, cudaStream_t s) {
  using C = TrsvCfg<T, RCW>;
  constexpr int RC = C::RC;
  constexpr size_t smem = trsvl_smem_bytes<T, kNB, RC, C::NS>();
  auto kern = k_trsv_left<T, kNB, RC, UPPER, C::NS, C::MINB, XV>;
  static int resident = [&] {
    int dev = 0, sms = 0, per_sm = 0;
    if (set_smem(kern, (int)smem) != cudaSuccess) return 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
    return sms * per_sm;
  }();
  const int nblk = ceil_div(n, kNB), nchunk = ceil_div(nrhs, RC);
  if (resident < nchunk) return EBV_ERR_UNSUPPORTED;
  const int G = std::max(1, std::min(resident / nchunk, nblk));
  EBV_CU(cudaMemsetAsync(xw, 0, sizeof(unsigned long long) * (size_t)nchunk * nblk * kNB * RC * XWords<T>::W, s));
  prof::Scope ps(s, prof::kTrsv, (double)n * n * nrhs);  // nominal n^2 flops per right-hand side
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(G * nchunk));
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  EBV_CU(cudaLaunchKernelEx(&cfg, kern, F, n, B, ldb, nrhs, dinv, xw, st));
  return launch_ok();
}

template <typename T, bool UPPER, bool XV>
ebv_status_t trsv_one(MatView<T, XV> F, int64_t n, T *B, int64_t ldb, int nrhs, const T *dinv,
                      unsigned long long *xw, DevStatus *st, cudaStream_t s) {
  // Chunk width: narrower chunks are independent chains with a smaller
  // coupling product per step.  FP64 up to 8 right-hand sides: chunks of 4
  // (an FP64 warp instruction costs the same whatever its active lanes, so
  // the product's instruction count is what to cut); 9..32 in chunks of 16
  // (measured at n = 16384, 32 RHS, binary32: 3.0 ms for the four triangle
  // solves against 3.8 in one chunk of 32 and 3.6 in four of 8).
  if (sizeof(T) == 8 && nrhs <= 8) return trsv_launch<T, UPPER, 4, XV>(F, n, B, ldb, nrhs, dinv, xw, st, s);
  if (nrhs <= 8) return trsv_launch<T, UPPER, 8, XV>(F, n, B, ldb, nrhs, dinv, xw, st, s);
  if (nrhs <= 32) return trsv_launch<T, UPPER, 16, XV>(F, n, B, ldb, nrhs, dinv, xw, st, s);
  return trsv_launch<T, UPPER, 32, XV>(F, n, B, ldb, nrhs, dinv, xw, st, s);
}

// Forward then backward block substitution of B (n x nrhs, T) in place.
template <typename T, bool XV>
ebv_status_t trsv_pair(MatView<T, XV> F, int64_t n, T *B, int64_t ldb, int nrhs, const T *dinv,
                       unsigned long long *xw, DevStatus *st, cudaStream_t s) {
  EBV_TRY((trsv_one<T, false, XV>(F, n, B, ldb, nrhs, dinv, xw, st, s)));
  return trsv_one<T, true, XV>(F, n, B, ldb, nrhs, dinv, xw, st, s);
}

// ---------------------------------------------------------------------------
// Solve with optional refinement.  Shared by the dense and banded paths
// through the factor view F and the residual callback.
// ---------------------------------------------------------------------------
template <typename T, bool XV, typename ResidualFn>
ebv_status_t solve_refined(MatView<T, XV> F, int64_t n, void *b, int64_t nrhs, int64_t ldb, const ebv_refine_t *refine,
                           ebv_refine_report_t *rep, char *w, const DenseSolveLayout &L, bool b_is_double,
                           ResidualFn residual, cudaStream_t s) {
  DevStatus *st = (DevStatus *)w;
  const int nr = (int)nrhs;
  T *dinv = (T *)(w + L.dinv);
  static const bool carveout = (set_smem(k_narrow<T>, 0), set_smem(k_update_x<T>, 0), set_smem(k_colmax, 0),
                                set_smem(k_ir_check, 0), set_smem(k_split_x, 0), true);
  (void)carveout;
  unsigned long long *xw = (unsigned long long *)(w + L.xw);
  EBV_TRY(diag_inverses<T>(F, n, dinv, s));
  if (!refine) {
    if (b_is_double == (sizeof(T) == 8)) return trsv_pair<T>(F, n, (T *)b, ldb, nr, dinv, xw, st, s);
    // FP32 factors applied to FP64 right-hand sides (mixed precisions, no refinement).
    T *c = (T *)(w + L.corr);
    k_narrow<T><<<grid_for(n * nrhs), 256, 0, s>>>((const double *)b, ldb, c, nrhs, n, nr, st);
    EBV_TRY(launch_ok());
    EBV_TRY(trsv_pair<T>(F, n, c, nrhs, nr, dinv, xw, st, s));
    k_update_x<T><<<grid_for(n * nrhs), 256, 0, s>>>((double *)b, ldb, c, nrhs, n, nr, 0, st);
    return launch_ok();
  }
  if (!b_is_double) return EBV_ERR_UNSUPPORTED;
  double *x = (double *)b;
  double *bsave = (double *)(w + L.bsave);
  double *r = (double *)(w + L.r);
  T *c = (T *)(w + L.corr);
  float *xhi = (float *)(w + L.xhi), *xlo = (float *)(w + L.xlo);
  unsigned long long *rmax = (unsigned long long *)(w + L.rmax), *bmax = (unsigned long long *)(w + L.bmax);
  EBV_CU(cudaMemcpy2DAsync(bsave, nrhs * 8, x, ldb * 8, nrhs * 8, n, cudaMemcpyDeviceToDevice, s));
  EBV_CU(cudaMemsetAsync(bmax, 0, nrhs * 8, s));
  k_colmax<<<grid_for(n * nrhs), 256, 0, s>>>(bsave, nrhs, n, nr, bmax);
  EBV_TRY(launch_ok());
  // x0 from the factors.
  k_narrow<T><<<grid_for(n * nrhs), 256, 0, s>>>(bsave, nrhs, c, nrhs, n, nr, st);
  EBV_TRY(launch_ok());
  EBV_TRY(trsv_pair<T>(F, n, c, nrhs, nr, dinv, xw, st, s));
  k_update_x<T><<<grid_for(n * nrhs), 256, 0, s>>>(x, ldb, c, nrhs, n, nr, 0, st);
  EBV_TRY(launch_ok());
  const int max_iter = std::max(0, refine->max_iter);
  for (int it = 0; it <= max_iter; ++it) {
    EBV_CU(cudaMemsetAsync(rmax, 0, nrhs * 8, s));
    EBV_TRY(residual(x, ldb, xhi, xlo, bsave, r, rmax, st, it == 0));
    k_ir_check<<<1, 1, 0, s>>>(rmax, bmax, nr, it, max_iter, refine->tol, st, rep);
    EBV_TRY(launch_ok());
    if (it == max_iter) break;
    k_narrow<T><<<grid_for(n * nrhs), 256, 0, s>>>(r, nrhs, c, nrhs, n, nr, st);
    EBV_TRY(launch_ok());
    EBV_TRY(trsv_pair<T>(F, n, c, nrhs, nr, dinv, xw, st, s));
    k_update_x<T><<<grid_for(n * nrhs), 256, 0, s>>>(x, ldb, c, nrhs, n, nr, 1, st);
    EBV_TRY(launch_ok());
  }
  return EBV_OK;
}

}  // namespace
}  // namespace ebv
