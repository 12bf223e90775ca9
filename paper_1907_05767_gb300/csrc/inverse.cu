// Product-form inverse (Eq. 4c): A^{-1} = U^{-1} L^{-1} from the packed
// Doolittle factors.  Eq. 4c writes the inverse as the product of the
// elimination's elementary transformations; grouped by 64-column blocks and
// then by halves, those products become
//   leaves   L_bb^{-1}, U_bb^{-1} of every 64 x 64 diagonal block (one CTA each),
//   levels   for a node [L11 0; L21 L22] (and its upper twin) whose halves are
//            already inverted:  Z21 = -Z22 (L21 Z11),  W12 = -(W11 U12) W22,
//   product  A^{-1} = W Z with W = U^{-1} (upper) and Z = L^{-1} (unit lower).
// The tree is bottom-up over aligned groups of 2^l blocks, so every level is
// two launches (the inner product, then the outer one) over all of its nodes
// and the whole inverse is 2 + 2*ceil(log2(n/64)) launches.  W and Z are kept
// packed like the factors (Z strictly below the diagonal, W on and above) in
// the workspace; the inner products of a level are parked in the caller's
// output, which is free until the final product overwrites it.
//
// Every product is a SIMT tile product in the working precision (FP64 has no
// fast tensor-core path on this GPU); the triangles are skipped at tile
// granularity: a tile's k-range stops where its triangular operand is zero.
// Work: 4n^3/3 flops in all (n^3/3 per triangle inverse, 2n^3/3 for W Z).
#include "dense_kernels.cuh"
#include "internal.h"

namespace ebv {
namespace {

template <typename T>
struct InvTile;
template <>
struct InvTile<double> {
  static constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
};
template <>
struct InvTile<float> {
  static constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
};

enum : int { kFull = 0, kUnitLower = 1, kUpper = 2 };

// Operand element (r, c) at p[r*ld + c], read through its triangle: a unit
// lower operand has ones on the diagonal and zeros above it, an upper one
// zeros below the diagonal.
template <typename T>
struct Opnd {
  const T *p;
  int64_t ld;
  int mode;
  __device__ __forceinline__ T at(int64_t r, int64_t c) const {
    if (mode == kUnitLower) return c < r ? p[r * ld + c] : (c == r ? T(1) : T(0));
    if (mode == kUpper) return c >= r ? p[r * ld + c] : T(0);
    return p[r * ld + c];
  }
};

template <typename T, int BM, int BN, int BK, int NT>
struct Slab {
  static constexpr int NA = BM * BK / NT, NB_ = BK * BN / NT;
  T a[NA], b[NB_];
};

// C(bm + i, bn + j) = alpha * sum_{k in [kb, ke)} A(bm + i, k) B(k, bn + j)
// for the CTA's BM x BN tile; rows >= M, columns >= N read as zero.  The next
// k-slab's global loads are in flight while the current one is multiplied.
template <typename T, int BM, int BN, int BK, int TM, int TN>
__device__ __forceinline__ void tile_product(const Opnd<T> &A, const Opnd<T> &B, int64_t bm, int64_t bn, int64_t M,
                                             int64_t N, int64_t kb, int64_t ke, T alpha, T *C, int64_t ldc) {
  constexpr int NTX = BN / TN, NTY = BM / TM, NT = NTX * NTY;
  static_assert((BM * BK) % NT == 0 && (BK * BN) % NT == 0, "slab must divide evenly");
  __shared__ T As[2][BK][BM + 1];
  __shared__ T Bs[2][BK][BN + 1];
  const int tx = threadIdx.x % NTX, ty = threadIdx.x / NTX;
  Slab<T, BM, BN, BK, NT> sl;
  auto fetch = [&](int64_t kk) {
#pragma unroll
    for (int q = 0; q < Slab<T, BM, BN, BK, NT>::NA; ++q) {
      const int e = threadIdx.x + NT * q, i = e / BK, k = e % BK;
      const int64_t gi = bm + i, gk = kk + k;
      sl.a[q] = (gi < M && gk < ke) ? A.at(gi, gk) : T(0);
    }
#pragma unroll
    for (int q = 0; q < Slab<T, BM, BN, BK, NT>::NB_; ++q) {
      const int e = threadIdx.x + NT * q, k = e / BN, j = e % BN;
      const int64_t gk = kk + k, gj = bn + j;
      sl.b[q] = (gk < ke && gj < N) ? B.at(gk, gj) : T(0);
    }
  };
  auto put = [&](int buf) {
#pragma unroll
    for (int q = 0; q < Slab<T, BM, BN, BK, NT>::NA; ++q) {
      const int e = threadIdx.x + NT * q;
      As[buf][e % BK][e / BK] = sl.a[q];
    }
#pragma unroll
    for (int q = 0; q < Slab<T, BM, BN, BK, NT>::NB_; ++q) {
      const int e = threadIdx.x + NT * q;
      Bs[buf][e / BN][e % BN] = sl.b[q];
    }
  };
  T acc[TM][TN];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) acc[a][b] = T(0);
  int buf = 0;
  if (kb < ke) {
    fetch(kb);
    put(0);
  }
  __syncthreads();
  for (int64_t kk = kb; kk < ke; kk += BK) {
    const bool more = kk + BK < ke;
    if (more) fetch(kk + BK);
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      T ra[TM], rb[TN];
#pragma unroll
      for (int a = 0; a < TM; ++a) ra[a] = As[buf][k][ty + a * NTY];
#pragma unroll
      for (int b = 0; b < TN; ++b) rb[b] = Bs[buf][k][tx + b * NTX];
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b) acc[a][b] = fma(ra[a], rb[b], acc[a][b]);
    }
    if (more) put(buf ^ 1);  // the other buffer was last read before the previous barrier
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int a = 0; a < TM; ++a) {
    const int64_t gi = bm + ty + a * NTY;
    if (gi >= M) continue;
#pragma unroll
    for (int b = 0; b < TN; ++b) {
      const int64_t gj = bn + tx + b * NTX;
      if (gj < N) C[gi * ldc + gj] = alpha * acc[a][b];
    }
  }
}

// Leaves: the inverses of the triangles of every 64 x 64 diagonal block, into
// the packed W\Z array P (Z_bb strictly below the diagonal, W_bb on and above).
// A ragged last block is padded with the identity, whose inverse it keeps.
// Dynamic shared memory: diag_smem_bytes<T, kNB>().
template <typename T>
__global__ void __launch_bounds__(4 * kNB) k_inv_leaf(MatView<T> F, int64_t n, T *P, int64_t ldp) {
  constexpr int NB = kNB, NT = 4 * kNB;
  extern __shared__ __align__(16) unsigned char dsm[];
  T(*D)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(dsm);
  T *LT = reinterpret_cast<T *>(dsm + sizeof(T) * NB * (NB + 1));
  T *VT = LT + NB * diag_tstride<T, NB>();
  T *buf = VT + NB * diag_tstride<T, NB>();
  __shared__ T rcp[NB];
  const int64_t i0 = (int64_t)blockIdx.x * NB;
  const int hb = (int)min64(NB, n - i0);
  stage_tile<NB, NT, NB + 1>(&D[0][0], [&](int r, int k) {
    return (r < hb && k < hb) ? F.get(i0 + r, i0 + k) : (r == k ? T(1) : T(0));
  });
  __syncthreads();
  for (int r = threadIdx.x; r < NB; r += NT) rcp[r] = pivot_rcp(D[r][r]);
  __syncthreads();
  masked_factor_copies<T, NB, NT>(D, rcp, LT, VT);
  __syncthreads();
  // The sweeps read LT / VT for the last time before their final barrier, so
  // the two inverses (2 * NB * NB elements) may overwrite them.
  static_assert(2 * NB * NB <= 2 * NB * diag_tstride<T, NB>(), "inverses must fit over LT and VT");
  T *inv = LT;
  triangle_inverses<T, NB, NT>(LT, VT, buf, rcp, inv);
  __syncthreads();
  for (int e = threadIdx.x; e < NB * NB; e += NT) {
    const int r = e / NB, c = e % NB;
    if (r < hb && c < hb) P[(i0 + r) * ldp + i0 + c] = r > c ? inv[r * NB + c] : inv[NB * NB + r * NB + c];
  }
}

// One level of the tree: nodes of span 2h at offsets o = z*2h whose second
// half [o+h, o+h+n2) is not empty (n2 = min(h, n-o-h)).  blockIdx.z = 2*node +
// side, side 0 the lower triangle, 1 the upper.
//   STAGE 1:  T_L = L21 Z11 (n2 x h)  and  T_U = W11 U12 (h x n2), into x.
//   STAGE 2:  Z21 = -Z22 T_L  and  W12 = -T_U W22, into P.
template <typename T, int STAGE>
__global__ void __launch_bounds__((InvTile<T>::BM / InvTile<T>::TM) * (InvTile<T>::BN / InvTile<T>::TN))
    k_inv_level(const T *lu, int64_t ldl, T *P, int64_t ldp, T *x, int64_t ldx, int64_t n, int64_t h) {
  using G = InvTile<T>;
  const int64_t node = blockIdx.z >> 1, o = node * 2 * h;
  const int side = blockIdx.z & 1;
  const int64_t n2 = min64(h, n - o - h);
  const int64_t bm = (int64_t)blockIdx.y * G::BM, bn = (int64_t)blockIdx.x * G::BN;
  const int64_t M = side == 0 ? n2 : h, N = side == 0 ? h : n2;
  if (bm >= M || bn >= N) return;  // the whole CTA: before any barrier
  T *p_lo = P + (o + h) * ldp + o, *p_up = P + o * ldp + o + h;  // Z21 / W12 positions
  if (STAGE == 1) {
    if (side == 0) {  // T_L(i, j) = sum_{k >= j} L21(i, k) Z11(k, j)
      const Opnd<T> A{lu + (o + h) * ldl + o, ldl, kFull}, B{P + o * ldp + o, ldp, kUnitLower};
      tile_product<T, G::BM, G::BN, G::BK, G::TM, G::TN>(A, B, bm, bn, M, N, bn, h, T(1), x + (o + h) * ldx + o, ldx);
    } else {  // T_U(i, j) = sum_{k >= i} W11(i, k) U12(k, j)
      const Opnd<T> A{P + o * ldp + o, ldp, kUpper}, B{lu + o * ldl + o + h, ldl, kFull};
      tile_product<T, G::BM, G::BN, G::BK, G::TM, G::TN>(A, B, bm, bn, M, N, bm, h, T(1), x + o * ldx + o + h, ldx);
    }
  } else {
    const T *pd = P + (o + h) * ldp + o + h;  // Z22 \ W22
    if (side == 0) {  // Z21(i, j) = -sum_{k <= i} Z22(i, k) T_L(k, j)
      const Opnd<T> A{pd, ldp, kUnitLower}, B{x + (o + h) * ldx + o, ldx, kFull};
      tile_product<T, G::BM, G::BN, G::BK, G::TM, G::TN>(A, B, bm, bn, M, N, 0, min64(bm + G::BM, n2), T(-1),
                                                         p_lo, ldp);
    } else {  // W12(i, j) = -sum_{k <= j} T_U(i, k) W22(k, j)
      const Opnd<T> A{x + o * ldx + o + h, ldx, kFull}, B{pd, ldp, kUpper};
      tile_product<T, G::BM, G::BN, G::BK, G::TM, G::TN>(A, B, bm, bn, M, N, 0, min64(bn + G::BN, n2), T(-1),
                                                         p_up, ldp);
    }
  }
}

// X = W Z: X(i, j) = sum_{k >= max(i, j)} W(i, k) Z(k, j).  One CTA per tile,
// tiles taken shell by shell (shell m: the tiles with max(I, J) = m, whose
// k-range is the longest for m = 0), so the long tiles start first.
template <typename T>
__global__ void __launch_bounds__((InvTile<T>::BM / InvTile<T>::TM) * (InvTile<T>::BN / InvTile<T>::TN))
    k_inv_product(const T *P, int64_t ldp, T *x, int64_t ldx, int64_t n) {
  using G = InvTile<T>;
  static_assert(G::BM == G::BN, "square tiles");
  const int64_t b = blockIdx.x;
  int64_t m = (int64_t)sqrt((double)b);
  while (m * m > b) --m;
  while ((m + 1) * (m + 1) <= b) ++m;
  const int64_t t = b - m * m;  // 0 .. 2m
  const int64_t I = t <= m ? m : t - m - 1, J = t <= m ? t : m;
  const int64_t bm = I * G::BM, bn = J * G::BN;
  const Opnd<T> W{P, ldp, kUpper}, Z{P, ldp, kUnitLower};
  tile_product<T, G::BM, G::BN, G::BK, G::TM, G::TN>(W, Z, bm, bn, n, n, max64(bm, bn), n, T(1), x, ldx);
}

inline int64_t inv_ldp(int64_t n) { return (n + 3) / 4 * 4; }

template <typename T>
ebv_status_t inverse_t(int64_t n, const T *lu, int64_t ldl, T *x, int64_t ldx, void *ws, cudaStream_t s) {
  using G = InvTile<T>;
  constexpr int NT = (G::BM / G::TM) * (G::BN / G::TN);
  if (n == 0) return EBV_OK;
  static const cudaError_t attr = [] {  // once per process and type (thread-safe static initialisation)
    cudaError_t e = set_smem(k_inv_leaf<T>, (int)diag_smem_bytes<T, kNB>());
    if (e == cudaSuccess) e = set_smem(k_inv_level<T, 1>, 0);
    if (e == cudaSuccess) e = set_smem(k_inv_level<T, 2>, 0);
    if (e == cudaSuccess) e = set_smem(k_inv_product<T>, 0);
    return e;
  }();
  if (attr != cudaSuccess) return EBV_ERR_CUDA;
  T *P = static_cast<T *>(ws);
  const int64_t ldp = inv_ldp(n);
  const int64_t nblk = ceil_div(n, kNB);
  {
    prof::Scope ps(s, prof::kInverse, 4.0 * kNB * kNB * kNB / 3.0 * nblk);
    k_inv_leaf<T><<<(unsigned)nblk, 4 * kNB, diag_smem_bytes<T, kNB>(), s>>>(dense_view(const_cast<T *>(lu), ldl),
                                                                             n, P, ldp);
    EBV_TRY(launch_ok());
  }
  for (int64_t h = kNB; h < n; h *= 2) {
    const int64_t nodes = (n - h + 2 * h - 1) / (2 * h);  // nodes whose second half is not empty
    const double work = 2.0 * (double)h * (double)h * (double)(n - nodes * h);  // ~ n2 h^2 per side and stage
    const dim3 grid(ceil_div(h, G::BN), ceil_div(h, G::BM), (unsigned)(2 * nodes));
    {
      prof::Scope ps(s, prof::kInverse, work);
      k_inv_level<T, 1><<<grid, NT, 0, s>>>(lu, ldl, P, ldp, x, ldx, n, h);
      EBV_TRY(launch_ok());
    }
    {
      prof::Scope ps(s, prof::kInverse, work);
      k_inv_level<T, 2><<<grid, NT, 0, s>>>(lu, ldl, P, ldp, x, ldx, n, h);
      EBV_TRY(launch_ok());
    }
  }
  const int64_t nt = ceil_div(n, G::BM);
  prof::Scope ps(s, prof::kInverse, 2.0 * (double)n * n * n / 3.0);
  k_inv_product<T><<<(unsigned)(nt * nt), NT, 0, s>>>(P, ldp, x, ldx, n);
  return launch_ok();
}

}  // namespace

size_t inverse_ws(int64_t n, ebv_prec_t prec) {
  const size_t es = prec == EBV_FP64 ? 8 : 4;
  return n > 0 ? align256((size_t)n * (size_t)inv_ldp(n) * es) : 0;
}

ebv_status_t inverse(int64_t n, ebv_prec_t prec, const void *lu, int64_t ldl, void *x, int64_t ldx, void *ws,
                     cudaStream_t s) {
  if (prec == EBV_FP64)
    return inverse_t<double>(n, static_cast<const double *>(lu), ldl, static_cast<double *>(x), ldx, ws, s);
  return inverse_t<float>(n, static_cast<const float *>(lu), ldl, static_cast<float *>(x), ldx, ws, s);
}

}  // namespace ebv
