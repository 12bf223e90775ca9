// Adjoint of X = A^{-1} B for a batch of equal-size FP64 systems (project
// addition; the paper has no gradients).  With the stored factors A = LU,
// A^T = U^T L^T, so for dLoss/dX = G:
//   grad_B = A^{-T} G : U^T z = G (forward, non-unit diagonal through FP64
//                       reciprocals), then L^T w = z (backward, unit), w = grad_B;
//   grad_A = -grad_B X^T (an outer product with nrhs terms per entry; on this
//                       GPU the FP64 multiply-adds, not the n x n output,
//                       bound it).
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

// The same solve with Z resident in shared memory (n x NR doubles, columns
// >= nrhs zero) for systems whose right-hand sides fit on chip.  Per 32-row
// block, warp 0 solves the diagonal block in registers: lane p holds row p
// of Z and column p of the block of U (resp. L), the pivot reciprocals are
// taken all at once, and each of the 32 steps is NR shuffles plus NR fused
// multiply-adds.  Then every thread updates whole rows below (resp. above)
// against the finished block: the factor rows are read coalesced and the
// block of Z is a shared-memory broadcast.
// Dynamic shared memory: n * NR * sizeof(double).
template <int NR>
__global__ void __launch_bounds__(AT, 2) k_adjoint_solve_smem(int64_t n, int nrhs, const double *lu, int64_t lda,
                                                              int64_t stride_lu, double *z_all) {
  extern __shared__ double zs[];
  const double *F = lu + (int64_t)blockIdx.x * stride_lu;
  double *Z = z_all + (int64_t)blockIdx.x * n * nrhs;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t e = threadIdx.x; e < n * NR; e += AT) {
    const int64_t i = e / NR;
    const int c = (int)(e % NR);
    zs[e] = c < nrhs ? Z[i * nrhs + c] : 0.0;
  }
  __syncthreads();
  // U^T z = g: blocks in increasing order.
  for (int64_t k0 = 0; k0 < n; k0 += ANB) {
    const int w = (int)min64(ANB, n - k0);
    if (warp == 0) {
      const bool act = lane < w;
      double u[ANB], z[NR];
#pragma unroll
      for (int r = 0; r < ANB; ++r) u[r] = (act && r < w) ? F[(k0 + r) * lda + k0 + lane] : 0.0;  // U[r][lane]
      const double rc = act ? 1.0 / F[(k0 + lane) * lda + k0 + lane] : 0.0;
#pragma unroll
      for (int c = 0; c < NR; ++c) z[c] = act ? zs[(k0 + lane) * NR + c] : 0.0;
#pragma unroll
      for (int r = 0; r < ANB; ++r) {
        if (r < w) {
#pragma unroll
          for (int c = 0; c < NR; ++c) {
            if (lane == r) z[c] *= rc;  // z_r is final
            const double zr = __shfl_sync(0xffffffffu, z[c], r);
            if (lane > r) z[c] -= u[r] * zr;  // z_p -= U^T[p][r] z_r = U[r][p] z_r
          }
        }
      }
#pragma unroll
      for (int c = 0; c < NR; ++c)
        if (act) zs[(k0 + lane) * NR + c] = z[c];
    }
    __syncthreads();
    for (int64_t i = k0 + w + threadIdx.x; i < n; i += AT) {
      double acc[NR];
#pragma unroll
      for (int c = 0; c < NR; ++c) acc[c] = zs[i * NR + c];
#pragma unroll 8
      for (int r = 0; r < w; ++r) {
        const double f = F[(k0 + r) * lda + i];
#pragma unroll
        for (int c = 0; c < NR; ++c) acc[c] -= f * zs[(k0 + r) * NR + c];
      }
#pragma unroll
      for (int c = 0; c < NR; ++c) zs[i * NR + c] = acc[c];
    }
    __syncthreads();
  }
  // L^T w = z: blocks in decreasing order, unit diagonal.
  for (int64_t kend = n; kend > 0; kend -= ANB) {
    const int64_t k0 = max64(0, kend - ANB);
    const int w = (int)(kend - k0);
    if (warp == 0) {
      const bool act = lane < w;
      double l[ANB], z[NR];
#pragma unroll
      for (int r = 0; r < ANB; ++r) l[r] = (act && r < w) ? F[(k0 + r) * lda + k0 + lane] : 0.0;  // L[r][lane]
#pragma unroll
      for (int c = 0; c < NR; ++c) z[c] = act ? zs[(k0 + lane) * NR + c] : 0.0;
#pragma unroll
      for (int r = ANB - 1; r >= 1; --r) {
        if (r < w) {
#pragma unroll
          for (int c = 0; c < NR; ++c) {
            const double zr = __shfl_sync(0xffffffffu, z[c], r);
            if (lane < r) z[c] -= l[r] * zr;  // z_p -= L^T[p][r] z_r = L[r][p] z_r
          }
        }
      }
#pragma unroll
      for (int c = 0; c < NR; ++c)
        if (act) zs[(k0 + lane) * NR + c] = z[c];
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < k0; i += AT) {
      double acc[NR];
#pragma unroll
      for (int c = 0; c < NR; ++c) acc[c] = zs[i * NR + c];
#pragma unroll 8
      for (int r = 0; r < w; ++r) {
        const double f = F[(k0 + r) * lda + i];
#pragma unroll
        for (int c = 0; c < NR; ++c) acc[c] -= f * zs[(k0 + r) * NR + c];
      }
#pragma unroll
      for (int c = 0; c < NR; ++c) zs[i * NR + c] = acc[c];
    }
    __syncthreads();
  }
  for (int64_t e = threadIdx.x; e < n * nrhs; e += AT) Z[e] = zs[(e / nrhs) * NR + e % nrhs];
}

constexpr size_t kAdjSmemMax = 100 * 1024;  // two CTAs per SM

// grad_A(i, j) = -sum_c grad_B(i, c) X(j, c); CTA (AROWS-row tile, system).
// X of the system (n x nrhs) and the tile's rows of grad_B (AROWS x NR,
// zero-padded) are staged in shared memory once per CTA; each thread takes columns j
// (coalesced streaming stores) and, per column, all AROWS rows unrolled:
// AROWS independent NR-term FP64 dot products.
constexpr int AROWS = 32;
constexpr int AMAXRHS = 16;

template <int NR>
__global__ void __launch_bounds__(AT) k_adjoint_outer(int64_t n, int nrhs, const double *gb_all, const double *x_all,
                                                      double *ga_all) {
  extern __shared__ double xs[];  // n x nrhs, then AROWS x NR
  const int64_t sys = blockIdx.y;
  const double *X = x_all + sys * n * nrhs;
  const double *GB = gb_all + sys * n * nrhs;
  double *GA = ga_all + sys * n * n;
  const int64_t r0 = (int64_t)blockIdx.x * AROWS;
  const int rows = (int)min64(AROWS, n - r0);
  double *gbs = xs + n * nrhs;
  for (int64_t e = threadIdx.x; e < n * nrhs; e += AT) xs[e] = X[e];
  for (int e = threadIdx.x; e < AROWS * NR; e += AT) {
    const int ii = e / NR, c = e % NR;
    gbs[e] = (ii < rows && c < nrhs) ? GB[(r0 + ii) * nrhs + c] : 0.0;
  }
  __syncthreads();
  for (int64_t j = threadIdx.x; j < n; j += AT) {
    double xj[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) xj[c] = c < nrhs ? xs[j * nrhs + c] : 0.0;
#pragma unroll
    for (int ii = 0; ii < AROWS; ++ii) {
      if (ii < rows) {
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < NR; ++c) s = fma(gbs[ii * NR + c], xj[c], s);
        __stcs(&GA[(r0 + ii) * n + j], -s);
      }
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
  const int nr = nrhs <= 4 ? 4 : nrhs <= 8 ? 8 : 16;
  const size_t outer_smem = sizeof(double) * ((size_t)n * nrhs + AROWS * nr);
  if (grad_a && outer_smem > 200 * 1024) return EBV_ERR_UNSUPPORTED;  // X of one system must fit on chip
  if (nrhs == 0) {  // grad_B is empty and grad_A = 0
    if (grad_a) EBV_CU(cudaMemsetAsync(grad_a, 0, sizeof(double) * (size_t)batch * n * n, (cudaStream_t)stream));
    return EBV_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  EBV_CU(cudaMemcpyAsync(grad_b, grad_x, sizeof(double) * (size_t)batch * n * nrhs, cudaMemcpyDeviceToDevice, s));
  {
    prof::Scope ps(s, prof::kAdjoint, 2.0 * batch * n * n * nrhs);
    const size_t zsm = sizeof(double) * (size_t)n * nr;
    if (zsm <= kAdjSmemMax) {
      static const cudaError_t attr4 = set_smem(k_adjoint_solve_smem<4>, (int)kAdjSmemMax);
      static const cudaError_t attr8 = set_smem(k_adjoint_solve_smem<8>, (int)kAdjSmemMax);
      static const cudaError_t attr16 = set_smem(k_adjoint_solve_smem<16>, (int)kAdjSmemMax);
      if (attr4 != cudaSuccess || attr8 != cudaSuccess || attr16 != cudaSuccess) return EBV_ERR_CUDA;
      if (nr == 4)
        k_adjoint_solve_smem<4><<<(unsigned)batch, AT, zsm, s>>>(n, (int)nrhs, lu, lda, stride_lu, grad_b);
      else if (nr == 8)
        k_adjoint_solve_smem<8><<<(unsigned)batch, AT, zsm, s>>>(n, (int)nrhs, lu, lda, stride_lu, grad_b);
      else
        k_adjoint_solve_smem<16><<<(unsigned)batch, AT, zsm, s>>>(n, (int)nrhs, lu, lda, stride_lu, grad_b);
    } else {
      k_adjoint_solve<<<(unsigned)batch, AT, 0, s>>>(n, (int)nrhs, lu, lda, stride_lu, grad_b);
    }
    EBV_TRY(launch_ok());
  }
  if (!grad_a) return EBV_OK;
  static const cudaError_t attr = [] {
    cudaError_t e = set_smem(k_adjoint_outer<4>, 200 * 1024);
    if (e == cudaSuccess) e = set_smem(k_adjoint_outer<8>, 200 * 1024);
    if (e == cudaSuccess) e = set_smem(k_adjoint_outer<16>, 200 * 1024);
    return e;
  }();
  if (attr != cudaSuccess) return EBV_ERR_CUDA;
  prof::Scope ps(s, prof::kOther, 2.0 * batch * n * n * nrhs);
  dim3 grid((unsigned)((n + AROWS - 1) / AROWS), (unsigned)batch);
  if (nr == 4)
    k_adjoint_outer<4><<<grid, AT, outer_smem, s>>>(n, (int)nrhs, grad_b, x, grad_a);
  else if (nr == 8)
    k_adjoint_outer<8><<<grid, AT, outer_smem, s>>>(n, (int)nrhs, grad_b, x, grad_a);
  else
    k_adjoint_outer<16><<<grid, AT, outer_smem, s>>>(n, (int)nrhs, grad_b, x, grad_a);
  return launch_ok();
}
