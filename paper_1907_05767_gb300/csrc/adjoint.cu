// Adjoint of X = A^{-1} B for a batch of equal-size FP64 systems (project
// addition; the paper has no gradients).  With the stored factors A = LU,
// A^T = U^T L^T, so for dLoss/dX = G:
//   grad_B = A^{-T} G : U^T z = G (forward, non-unit diagonal through FP64
//                       reciprocals), then L^T w = z (backward, unit), w = grad_B;
//   grad_A = -grad_B X^T (an outer product with nrhs terms per entry; the
//                       n x n output makes this step HBM-write-bound).
// Both triangles are read in their stored orientation: column i of U^T is row
// i of U, so the updates below a diagonal block read contiguous rows.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace ebv {
namespace {

constexpr int ANB = 32;   // block of the transposed substitutions
constexpr int AT = 256;   // threads per CTA

// One CTA per system: Z (n x nrhs, in place) = A^{-T} Z.
__global__ void __launch_bounds__(AT) k_adjoint_solve(int64_t n, int nrhs, const double *lu, int64_t lda,
                                                      int64_t stride_lu, double *z_all) {
  const double *F = lu + (int64_t)blockIdx.x * stride_lu;
  double *Z = z_all + (int64_t)blockIdx.x * n * nrhs;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // U^T z = g: blocks in increasing order.
  for (int64_t k0 = 0; k0 < n; k0 += ANB) {
    const int w = (int)min64(ANB, n - k0);
    if (warp == 0) {
      for (int r = 0; r < w; ++r) {
        double rc = 0.0;
        if (lane == 0) rc = 1.0 / F[(k0 + r) * lda + k0 + r];
        rc = __shfl_sync(0xffffffffu, rc, 0);
        for (int c = lane; c < nrhs; c += 32) Z[(k0 + r) * nrhs + c] *= rc;
        __syncwarp();
        // z_p -= U^T[p][r] z_r = U[r][p] z_r for p > r inside the block
        for (int e = lane; e < (w - 1 - r) * nrhs; e += 32) {
          const int p = r + 1 + e / nrhs, c = e % nrhs;
          Z[(k0 + p) * nrhs + c] -= F[(k0 + r) * lda + k0 + p] * Z[(k0 + r) * nrhs + c];
        }
        __syncwarp();
      }
    }
    __syncthreads();
    for (int64_t e = threadIdx.x; e < (n - k0 - w) * nrhs; e += AT) {
      const int64_t i = k0 + w + e / nrhs;
      const int c = (int)(e % nrhs);
      double s = Z[i * nrhs + c];
      for (int r = 0; r < w; ++r) s -= F[(k0 + r) * lda + i] * Z[(k0 + r) * nrhs + c];
      Z[i * nrhs + c] = s;
    }
    __syncthreads();
  }
  // L^T w = z: blocks in decreasing order, unit diagonal.
  for (int64_t kend = n; kend > 0; kend -= ANB) {
    const int64_t k0 = max64(0, kend - ANB);
    const int w = (int)(kend - k0);
    if (warp == 0) {
      for (int r = w - 1; r > 0; --r) {
        // z_p -= L^T[p][r] w_r = L[r][p] w_r for p < r inside the block
        for (int e = lane; e < r * nrhs; e += 32) {
          const int p = e / nrhs, c = e % nrhs;
          Z[(k0 + p) * nrhs + c] -= F[(k0 + r) * lda + k0 + p] * Z[(k0 + r) * nrhs + c];
        }
        __syncwarp();
      }
    }
    __syncthreads();
    for (int64_t e = threadIdx.x; e < k0 * nrhs; e += AT) {
      const int64_t i = e / nrhs;
      const int c = (int)(e % nrhs);
      double s = Z[i * nrhs + c];
      for (int r = 0; r < w; ++r) s -= F[(k0 + r) * lda + i] * Z[(k0 + r) * nrhs + c];
      Z[i * nrhs + c] = s;
    }
    __syncthreads();
  }
}

// grad_A(i, j) = -sum_c grad_B(i, c) X(j, c); CTA (row tile, system).  X of
// the system is staged in shared memory once per CTA; each thread writes a
// run of consecutive j (coalesced, streaming stores).
constexpr int AROWS = 16;
constexpr int AMAXRHS = 16;

__global__ void __launch_bounds__(AT) k_adjoint_outer(int64_t n, int nrhs, const double *gb_all, const double *x_all,
                                                      double *ga_all) {
  extern __shared__ double xs[];  // n x nrhs, then AROWS x nrhs
  const int64_t sys = blockIdx.y;
  const double *X = x_all + sys * n * nrhs;
  const double *GB = gb_all + sys * n * nrhs;
  double *GA = ga_all + sys * n * n;
  const int64_t r0 = (int64_t)blockIdx.x * AROWS;
  double *gbs = xs + n * nrhs;
  for (int64_t e = threadIdx.x; e < n * nrhs; e += AT) xs[e] = X[e];
  for (int e = threadIdx.x; e < AROWS * nrhs; e += AT) {
    const int64_t i = r0 + e / nrhs;
    gbs[e] = i < n ? GB[i * nrhs + e % nrhs] : 0.0;
  }
  __syncthreads();
  for (int64_t j = threadIdx.x; j < n; j += AT) {
    double xj[AMAXRHS];
#pragma unroll
    for (int c = 0; c < AMAXRHS; ++c) xj[c] = c < nrhs ? xs[j * nrhs + c] : 0.0;
    for (int ii = 0; ii < AROWS && r0 + ii < n; ++ii) {
      double s = 0.0;
#pragma unroll
      for (int c = 0; c < AMAXRHS; ++c)
        if (c < nrhs) s = fma(gbs[ii * nrhs + c], xj[c], s);
      __stcs(&GA[(r0 + ii) * n + j], -s);
    }
  }
}

}  // namespace
}  // namespace ebv

using namespace ebv;

extern "C" ebv_status_t ebv_solve_adjoint(int64_t batch, int64_t n, int64_t nrhs, const double *lu, int64_t lda,
                                          int64_t stride_lu, const double *x, const double *grad_x, double *grad_b,
                                          double *grad_a, ebv_stream_t stream) {
  if (batch < 0 || n < 0 || nrhs < 0 || batch > 65535) return EBV_ERR_ARG;
  if (batch == 0 || n == 0) return EBV_OK;
  if (lda < n || stride_lu < lda * (n - 1) + n || nrhs > AMAXRHS) return EBV_ERR_ARG;
  if (!lu || !grad_x || !grad_b || (grad_a && !x)) return EBV_ERR_ARG;
  for (const void *p : {(const void *)lu, (const void *)x, (const void *)grad_x, (const void *)grad_b,
                        (const void *)grad_a})
    if (p && ((uintptr_t)p % 8) != 0) return EBV_ERR_ARG;
  const size_t outer_smem = sizeof(double) * ((size_t)n * nrhs + AROWS * nrhs);
  if (grad_a && outer_smem > 200 * 1024) return EBV_ERR_UNSUPPORTED;  // X of one system must fit on chip
  if (nrhs == 0) {  // grad_B is empty and grad_A = 0
    if (grad_a) EBV_CU(cudaMemsetAsync(grad_a, 0, sizeof(double) * (size_t)batch * n * n, (cudaStream_t)stream));
    return EBV_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  EBV_CU(cudaMemcpyAsync(grad_b, grad_x, sizeof(double) * (size_t)batch * n * nrhs, cudaMemcpyDeviceToDevice, s));
  {
    prof::Scope ps(s, prof::kAdjoint, 2.0 * batch * n * n * nrhs);
    k_adjoint_solve<<<(unsigned)batch, AT, 0, s>>>(n, (int)nrhs, lu, lda, stride_lu, grad_b);
    EBV_TRY(launch_ok());
  }
  if (!grad_a) return EBV_OK;
  static const cudaError_t attr =
      set_smem(k_adjoint_outer, 200 * 1024);
  if (attr != cudaSuccess) return EBV_ERR_CUDA;
  prof::Scope ps(s, prof::kOther, 8.0 * batch * n * n);  // bytes written (HBM-bound step)
  dim3 grid((unsigned)((n + AROWS - 1) / AROWS), (unsigned)batch);
  k_adjoint_outer<<<grid, AT, outer_smem, s>>>(n, (int)nrhs, grad_b, x, grad_a);
  return launch_ok();
}
