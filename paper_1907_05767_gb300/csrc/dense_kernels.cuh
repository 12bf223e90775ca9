// Leaf kernels of the blocked / recursive Doolittle factorisation and the
// SIMT trailing-update GEMMs.  Used by the dense and the banded drivers.
//
// Method (arXiv 1907.05767): Eq. 6a divides the L vector of step r by the
// pivot; Eq. 6c subtracts the outer product of the L and U vectors from the
// trailing matrix; Eq. 7 pairs the long vector of step r with the short vector
// of step n-1-r so that every thread does the same amount of work.
#pragma once

#include "common.cuh"

namespace ebv {
namespace {  // internal linkage: every translation unit gets its own kernels

// Matrix view.  Element (i, j) lives at base[i*ld + j] when -kl <= j-i <= ku;
// elements outside that band read as 0 and are never written.  A dense matrix
// uses a huge band.  A row-band array ab (a_ij at ab[i*ldab + j-i+kl]) is the
// view base = ab + kl, ld = ldab - 1.
template <typename T>
struct MatView {
  T *base;
  int64_t ld;
  int64_t kl, ku;
  __device__ __forceinline__ bool in(int64_t i, int64_t j) const {
    const int64_t d = j - i;
    return d >= -kl && d <= ku;
  }
  __device__ __forceinline__ T get(int64_t i, int64_t j) const { return in(i, j) ? base[i * ld + j] : T(0); }
  __device__ __forceinline__ void put(int64_t i, int64_t j, T v) const {
    if (in(i, j)) base[i * ld + j] = v;
  }
};

constexpr int64_t kDenseBand = int64_t(1) << 60;

template <typename T>
inline MatView<T> dense_view(T *a, int64_t ld) { return MatView<T>{a, ld, kDenseBand, kDenseBand}; }
template <typename T>
inline MatView<T> band_view(T *ab, int64_t ldab, int64_t kl, int64_t ku) {
  return MatView<T>{ab + kl, ldab - 1, kl, ku};
}

// Low-precision shadow copies of the factors that feed the tensor-core GEMMs:
// lb (n x n, row-major) holds scale[0] * L, ut (n x n) holds scale[1] * U^T,
// so both GEMM operands are K-major.  Null when the trailing updates run in the
// working precision.
template <typename SH>
struct Shadow {
  SH *lb;
  SH *ut;
  int64_t ld;
  const float *scale;  // device: [sL, sU, 1/(sL*sU), -]
};

// ---------------------------------------------------------------------------
// Diagonal block: unblocked Doolittle on a w x w block (w <= NB), one CTA.
// Equal bi-vectorised ownership (Eq. 7): thread (p, g) owns the column pair
// {p, NB-1-p} -- one long and one short vector, so every pair meets the same
// number of rank-1 updates over the whole elimination -- and the rows
// g, g+NG, g+2NG, ...  The block lives in registers; each step broadcasts the
// pivot row, the pivot column and the FP64 pivot reciprocal through shared
// memory (double-buffered: one barrier per step).
// ---------------------------------------------------------------------------
template <typename T, int NB, int NT>
__global__ void __launch_bounds__(NT) k_diag_factor(MatView<T> A, int64_t k0, int w, int32_t *info) {
  constexpr int NP = NB / 2;
  constexpr int NG = NT / NP;
  constexpr int RPT = NB / NG;
  static_assert(NT % NP == 0 && NB % NG == 0, "shape");
  const int p = threadIdx.x % NP, g = threadIdx.x / NP;
  const int cj0 = p, cj1 = NB - 1 - p;
  __shared__ T rowbuf[2][NB];
  __shared__ T colbuf[2][NB];
  __shared__ double rcp[NB];
  __shared__ int bad;
  T v[RPT][2];
  if (threadIdx.x == 0) bad = NB;
#pragma unroll
  for (int t = 0; t < RPT; ++t) {
    const int i = g + NG * t;
    v[t][0] = (i < w && cj0 < w) ? A.get(k0 + i, k0 + cj0) : T(0);
    v[t][1] = (i < w && cj1 < w) ? A.get(k0 + i, k0 + cj1) : T(0);
  }
  __syncthreads();
  auto publish = [&](int r) {
    const int buf = r & 1;
#pragma unroll
    for (int t = 0; t < RPT; ++t) {
      const int i = g + NG * t;
      if (i >= w) continue;
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int j = s ? cj1 : cj0;
        if (j >= w) continue;
        if (i == r && j > r) rowbuf[buf][j] = v[t][s];
        if (j == r && i > r) colbuf[buf][i] = v[t][s];
        if (i == r && j == r) {
          const double pv = (double)v[t][s];
          rcp[r] = 1.0 / pv;
          if (!(pv != 0.0) || !isfinite(pv)) atomicMin(&bad, r);
        }
      }
    }
  };
  publish(0);
  __syncthreads();
  for (int r = 0; r < w; ++r) {
    const int buf = r & 1;
    const double rc = rcp[r];
#pragma unroll
    for (int t = 0; t < RPT; ++t) {
      const int i = g + NG * t;
      if (i > r && i < w) {
        const T l = (T)((double)colbuf[buf][i] * rc);  // Eq. 6a
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const int j = s ? cj1 : cj0;
          if (j == r)
            v[t][s] = l;
          else if (j > r && j < w)
            v[t][s] -= l * rowbuf[buf][j];  // Eq. 6c
        }
      }
    }
    if (r + 1 < w) publish(r + 1);
    __syncthreads();
  }
#pragma unroll
  for (int t = 0; t < RPT; ++t) {
    const int i = g + NG * t;
    if (i < w && cj0 < w) A.put(k0 + i, k0 + cj0, v[t][0]);
    if (i < w && cj1 < w) A.put(k0 + i, k0 + cj1, v[t][1]);
  }
  if (threadIdx.x == 0 && bad < NB && info) atomicCAS(info, 0, (int)(k0 + bad + 1));
}

// ---------------------------------------------------------------------------
// L21 = A21 U11^{-1}: the L vectors of the block's columns for all rows below
// it (Eq. 6a applied to rows r_begin..r_end-1).  Without pivoting every row is
// independent, so one thread owns one row (its w entries in registers) and U11
// is broadcast from shared memory.  Optionally writes the scaled low-precision
// shadow of L.
// ---------------------------------------------------------------------------
template <typename T, typename SH, int NB>
__global__ void __launch_bounds__(128) k_trsm_ru(MatView<T> A, int64_t k0, int w, int64_t r_begin, int64_t r_end,
                                                 Shadow<SH> sh) {
  __shared__ T U[NB][NB + 1];
  __shared__ double rc[NB];
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int i = e / NB, j = e % NB;
    U[i][j] = (i < w && j < w && j >= i) ? A.get(k0 + i, k0 + j) : T(0);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < NB; j += blockDim.x) rc[j] = j < w ? 1.0 / (double)U[j][j] : 0.0;
  __syncthreads();
  const int64_t i = r_begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= r_end) return;
  T v[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) v[j] = (j < w) ? A.get(i, k0 + j) : T(0);
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    v[j] = (T)((double)v[j] * rc[j]);
#pragma unroll
    for (int jj = j + 1; jj < NB; ++jj) v[jj] -= v[j] * U[j][jj];
  }
#pragma unroll
  for (int j = 0; j < NB; ++j)
    if (j < w) A.put(i, k0 + j, v[j]);
  if (sh.lb) {
    const float s = sh.scale[0];
    SH *dst = sh.lb + i * sh.ld + k0;
#pragma unroll
    for (int j = 0; j < NB; ++j)
      if (j < w) dst[j] = from_float<SH>((float)v[j] * s);
  }
}

// ---------------------------------------------------------------------------
// U12 = L11^{-1} A12: the U vectors of the block's rows for the columns
// c_begin..c_end-1 (unit lower forward substitution).  One thread owns one
// column; L11 is broadcast from shared memory.  Optionally writes the scaled
// low-precision shadow of U^T.
// ---------------------------------------------------------------------------
template <typename T, typename SH, int NB>
__global__ void __launch_bounds__(128) k_trsm_ll(MatView<T> A, int64_t r0, int h, int64_t c_begin, int64_t c_end,
                                                 Shadow<SH> sh) {
  __shared__ T L[NB][NB + 1];
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int i = e / NB, j = e % NB;
    L[i][j] = (i < h && j < i) ? A.get(r0 + i, r0 + j) : T(0);
  }
  __syncthreads();
  const int64_t j = c_begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= c_end) return;
  T v[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i) v[i] = (i < h) ? A.get(r0 + i, j) : T(0);
#pragma unroll
  for (int i = 0; i < NB; ++i) {
#pragma unroll
    for (int ii = i + 1; ii < NB; ++ii) v[ii] -= L[ii][i] * v[i];
  }
#pragma unroll
  for (int i = 0; i < NB; ++i)
    if (i < h) A.put(r0 + i, j, v[i]);
  if (sh.ut) {
    const float s = sh.scale[1];
    SH *dst = sh.ut + j * sh.ld + r0;
#pragma unroll
    for (int i = 0; i < NB; ++i)
      if (i < h) dst[i] = from_float<SH>((float)v[i] * s);
  }
}

// ---------------------------------------------------------------------------
// SIMT trailing update in the working precision (Eq. 6c aggregated over K
// steps):  A(m0+i, n0+j) -= sum_k A(m0+i, k0+k) * A(k0+k, n0+j).
// Register-tiled: each thread owns a TM x TN block of C.
// ---------------------------------------------------------------------------
template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    k_gemm_nn(MatView<T> A, int64_t m0, int64_t n0, int64_t k0, int64_t M, int64_t N, int64_t K) {
  constexpr int NTX = BN / TN, NTY = BM / TM, NT = NTX * NTY;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tx = threadIdx.x % NTX, ty = threadIdx.x / NTX;
  const int64_t bm = m0 + (int64_t)blockIdx.y * BM, bn = n0 + (int64_t)blockIdx.x * BN;
  const int64_t mend = m0 + M, nend = n0 + N, kend = k0 + K;
  T acc[TM][TN];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) acc[a][b] = T(0);
  for (int64_t kk = k0; kk < kend; kk += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += NT) {
      const int i = e / BK, k = e % BK;
      const int64_t gi = bm + i, gk = kk + k;
      As[k][i] = (gi < mend && gk < kend) ? A.get(gi, gk) : T(0);
    }
    for (int e = threadIdx.x; e < BK * BN; e += NT) {
      const int k = e / BN, j = e % BN;
      const int64_t gk = kk + k, gj = bn + j;
      Bs[k][j] = (gk < kend && gj < nend) ? A.get(gk, gj) : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      T ra[TM], rb[TN];
#pragma unroll
      for (int a = 0; a < TM; ++a) ra[a] = As[k][ty + a * NTY];
#pragma unroll
      for (int b = 0; b < TN; ++b) rb[b] = Bs[k][tx + b * NTX];
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b) acc[a][b] = fma(ra[a], rb[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < TM; ++a) {
    const int64_t gi = bm + ty + a * NTY;
    if (gi >= mend) continue;
#pragma unroll
    for (int b = 0; b < TN; ++b) {
      const int64_t gj = bn + tx + b * NTX;
      if (gj < nend && A.in(gi, gj)) {
        T *c = A.base + gi * A.ld + gj;
        *c = *c - acc[a][b];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// SIMT version of the mixed-precision update (reference path of the tensor-core
// kernel):  C(m0+i, n0+j) -= inv * sum_k lb(m0+i, k0+k) * ut(n0+j, k0+k),
// operands in bfloat16/half, products and sums in FP32.
// ---------------------------------------------------------------------------
template <typename SH, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    k_gemm_nt_simt(float *C, int64_t ldc, const SH *lb, const SH *ut, int64_t ldsh, const float *scale, int64_t m0,
                   int64_t n0, int64_t k0, int64_t M, int64_t N, int64_t K) {
  constexpr int NTX = BN / TN, NTY = BM / TM, NT = NTX * NTY;
  __shared__ float As[BK][BM + 1];
  __shared__ float Bs[BK][BN + 1];
  const int tx = threadIdx.x % NTX, ty = threadIdx.x / NTX;
  const int64_t bm = m0 + (int64_t)blockIdx.y * BM, bn = n0 + (int64_t)blockIdx.x * BN;
  const int64_t mend = m0 + M, nend = n0 + N, kend = k0 + K;
  float acc[TM][TN];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) acc[a][b] = 0.f;
  for (int64_t kk = k0; kk < kend; kk += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += NT) {
      const int i = e / BK, k = e % BK;
      const int64_t gi = bm + i, gk = kk + k;
      As[k][i] = (gi < mend && gk < kend) ? to_float(lb[gi * ldsh + gk]) : 0.f;
    }
    for (int e = threadIdx.x; e < BK * BN; e += NT) {
      const int j = e / BK, k = e % BK;
      const int64_t gk = kk + k, gj = bn + j;
      Bs[k][j] = (gk < kend && gj < nend) ? to_float(ut[gj * ldsh + gk]) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      float ra[TM], rb[TN];
#pragma unroll
      for (int a = 0; a < TM; ++a) ra[a] = As[k][ty + a * NTY];
#pragma unroll
      for (int b = 0; b < TN; ++b) rb[b] = Bs[k][tx + b * NTX];
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b) acc[a][b] = fmaf(ra[a], rb[b], acc[a][b]);
    }
    __syncthreads();
  }
  const float inv = scale[2];
#pragma unroll
  for (int a = 0; a < TM; ++a) {
    const int64_t gi = bm + ty + a * NTY;
    if (gi >= mend) continue;
#pragma unroll
    for (int b = 0; b < TN; ++b) {
      const int64_t gj = bn + tx + b * NTX;
      if (gj < nend) C[gi * ldc + gj] -= acc[a][b] * inv;
    }
  }
}

}  // namespace
}  // namespace ebv
