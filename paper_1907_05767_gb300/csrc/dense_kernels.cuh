// Leaf kernels of the blocked / recursive Doolittle factorisation and the
// SIMT trailing-update GEMMs.  Used by the dense and the banded host code.
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
// symlo: the factors of a symmetric band kept in its lower half only (L
// strictly below the diagonal, the pivots d on it; kl = ku): the U entries
// are read as u_ij = d_i l_ji (U = D L^T, the LDL^T form of Eq. 6a-b) and
// writes above the diagonal are dropped.  symraw (with symlo): entries above
// the diagonal read as a_ji instead -- the view of a still unfactored block.
//
// Profile (skyline) storage (plo set): per 64-block b, row block b keeps
// columns plo[b] .. 64b+63 (its lower part with the whole diagonal block),
// row-major with width 64(b+1) - plo[b], from base + poffL[b]; column block
// c keeps rows pup[c] .. 64c-1 (its part above the diagonal block),
// row-major with width 64, from base + poffU[c].  Entries outside read as 0
// and are never written; kl / ku bound the profile (the host loops' windows).
template <typename T, bool XV = false>
struct MatView {
  T *base;
  int64_t ld;
  int64_t kl, ku;
  // XV (compile time): the view may be symlo / symraw or profile storage.
  // The plain views (dense, row band) leave these fields unused, so their
  // kernels carry none of the extra index arithmetic.
  bool symlo = false;
  bool symraw = false;
  const int32_t *plo = nullptr, *pup = nullptr;
  const int64_t *poffL = nullptr, *poffU = nullptr;
  __device__ __forceinline__ bool in(int64_t i, int64_t j) const {
    const int64_t d = j - i;
    if (d < -kl || d > ku) return false;
    if constexpr (XV) {
      if (plo) {
        const int64_t b = i >> 6;
        return j < ((b + 1) << 6) ? j >= plo[b] : i >= pup[j >> 6];
      }
    }
    return true;
  }
  // Address of a stored element (in(i, j) must hold).
  __device__ __forceinline__ T *at(int64_t i, int64_t j) const {
    if constexpr (XV) {
      if (plo) {
        const int64_t b = i >> 6;
        if (j < ((b + 1) << 6)) {
          const int64_t lo = plo[b];
          return base + poffL[b] + (i - (b << 6)) * (((b + 1) << 6) - lo) + (j - lo);
        }
        const int64_t c = j >> 6;
        return base + poffU[c] + (i - pup[c]) * 64 + (j - (c << 6));
      }
    }
    return base + i * ld + j;
  }
  __device__ __forceinline__ T get(int64_t i, int64_t j) const {
    if (!in(i, j)) return T(0);
    if constexpr (XV) {
      if (symlo && j > i) return symraw ? base[j * ld + i] : base[j * ld + i] * base[i * ld + i];
    }
    return *at(i, j);
  }
  // The stored entry a_ij of an unfactored matrix (in(i, j) must hold); the
  // lower-half storages hold a_ij above the diagonal as a_ji.
  __device__ __forceinline__ T raw(int64_t i, int64_t j) const {
    if constexpr (XV) {
      if (symlo && j > i) return base[j * ld + i];
    }
    return *at(i, j);
  }
  __device__ __forceinline__ bool writable(int64_t i, int64_t j) const {
    if constexpr (XV) return in(i, j) && !(symlo && j > i);
    return in(i, j);
  }
  __device__ __forceinline__ void put(int64_t i, int64_t j, T v) const {
    if (writable(i, j)) *at(i, j) = v;
  }
};
// The views with lower-half symmetric or profile storage.
template <typename T>
using XView = MatView<T, true>;

constexpr int64_t kDenseBand = int64_t(1) << 60;

// Block envelope of a banded matrix, per 64-block of rows / columns (absolute
// indices): lo[b] = the first column holding a non-zero left of the diagonal
// in any row of row block b (none: a value >= the block's first row), up[b] =
// the first row holding a non-zero above the diagonal in any column of column
// block b.  Without row exchanges the factors stay inside the envelope (an L
// entry left of a row's first non-zero, or a U entry above a column's, never
// becomes non-zero), so for a panel ending at column kend the rows of block b
// carry no L entries when lo[b] >= kend, and the columns of block b no U
// entries when up[b] >= kend: their L21 / U12 tiles are zero and stay zero,
// and their trailing-update tiles receive nothing.  Null: no envelope.
struct Envelope {
  const int32_t *lo = nullptr;
  const int32_t *up = nullptr;
  __device__ __forceinline__ bool rows_empty(int64_t r, int64_t kend) const { return lo && lo[r / 64] >= kend; }
  __device__ __forceinline__ bool cols_empty(int64_t c, int64_t kend) const { return up && up[c / 64] >= kend; }
};

template <typename T>
inline MatView<T> dense_view(T *a, int64_t ld) { return MatView<T>{a, ld, kDenseBand, kDenseBand}; }
template <typename T>
inline MatView<T> band_view(T *ab, int64_t ldab, int64_t kl, int64_t ku) {
  return MatView<T>{ab + kl, ldab - 1, kl, ku};
}
// The lower triangle of a symmetric dense matrix (a_ij at a[i*ld + j], j <= i).
template <typename T>
inline XView<T> dense_symlo_view(T *a, int64_t ld) { return XView<T>{a, ld, kDenseBand, kDenseBand, true, false}; }
// The lower half of a symmetric band (a_ij at ab[i*ldab + j-i+kl], j <= i).
template <typename T>
inline XView<T> symlo_view(T *ab, int64_t ldab, int64_t kl) {
  return XView<T>{ab + kl, ldab - 1, kl, kl, true, false};
}

// Stage an NB x NB tile into shared memory (row stride S) with all of the
// thread's global loads issued before the first store, so one memory latency
// is paid instead of NB*NB/NT of them.  get(i, j) returns element (i, j).
// fetch_tile / put_tile are the two halves, for pipelines that keep the
// next tile's loads in flight while the current one is used.
template <int NB, int NT, typename T, typename Get>
__device__ __forceinline__ void fetch_tile(T (&r)[NB * NB / NT], Get get) {
  static_assert((NB * NB / NT) * NT == NB * NB, "tile must divide evenly");
#pragma unroll
  for (int q = 0; q < NB * NB / NT; ++q) {
    const int e = threadIdx.x + NT * q;
    r[q] = get(e / NB, e % NB);
  }
}
template <int NB, int NT, int S, typename T>
__device__ __forceinline__ void put_tile(T *dst, const T (&r)[NB * NB / NT]) {
#pragma unroll
  for (int q = 0; q < NB * NB / NT; ++q) {
    const int e = threadIdx.x + NT * q;
    dst[(e / NB) * S + e % NB] = r[q];
  }
}
template <int NB, int NT, int S, typename T, typename Get>
__device__ __forceinline__ void stage_tile(T *dst, Get get) {
  T r[NB * NB / NT];
  fetch_tile<NB, NT>(r, get);
  put_tile<NB, NT, S>(dst, r);
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
// Register-resident sweeps over one 64 x 64 diagonal block, one CTA of 256
// threads: lane p of warp g holds rows 8g .. 8g+7 of the column pair
// {p, NB-1-p} (the equal long/short pairing of Eq. 7).  triangle_inverses
// builds L11^{-1} and U11^{-1} from packed factors with one barrier per step
// (the substitution's preparation kernel uses it); the factorisation itself
// is the blocked kernel further down.
// Dynamic shared memory of the sweeps: diag_smem_bytes<T, NB>().
// ---------------------------------------------------------------------------
template <typename T, int NB>
__host__ __device__ constexpr int diag_tstride() { return NB + 16 / (int)sizeof(T); }  // 16-byte rows

template <typename T, int NB>
constexpr size_t diag_smem_bytes() {
  return sizeof(T) * ((size_t)NB * (NB + 1) + 2 * (size_t)NB * diag_tstride<T, NB>() + 4 * (size_t)NB);
}

template <typename T, int NB>
constexpr size_t pair_smem_bytes() { return 2 * sizeof(T) * NB * diag_tstride<T, NB>(); }

// Eight consecutive elements from 16-byte-aligned shared memory.
__device__ __forceinline__ void ld8(const float *p, float (&o)[8]) {
  const float4 a = reinterpret_cast<const float4 *>(p)[0], b = reinterpret_cast<const float4 *>(p)[1];
  o[0] = a.x, o[1] = a.y, o[2] = a.z, o[3] = a.w, o[4] = b.x, o[5] = b.y, o[6] = b.z, o[7] = b.w;
}
__device__ __forceinline__ void ld8(const double *p, double (&o)[8]) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const double2 a = reinterpret_cast<const double2 *>(p)[u];
    o[2 * u] = a.x, o[2 * u + 1] = a.y;
  }
}

// v[t] for a warp-uniform index t (a select chain: no local-memory array).
template <typename T, int N>
__device__ __forceinline__ T pick(const T (&v)[N], int t) {
  T r = v[0];
#pragma unroll
  for (int u = 1; u < N; ++u) r = (u == t) ? v[u] : r;
  return r;
}

// Transposed, masked copies of the packed factors for the inverse sweeps:
// LT[k][i] = l_ik (i > k, else 0) and VT[q][i] = u_iq / u_qq (i < q, else 0).
template <typename T, int NB, int NT>
__device__ __forceinline__ void masked_factor_copies(T (*D)[NB + 1], const T *rcp, T *LT, T *VT) {
  constexpr int TS = diag_tstride<T, NB>();
  for (int e = threadIdx.x; e < NB * NB; e += NT) {
    const int k = e / NB, i = e % NB;
    LT[k * TS + i] = i > k ? D[i][k] : T(0);
    VT[k * TS + i] = i < k ? D[i][k] * rcp[k] : T(0);
  }
}

// X = L^{-1} and Y = U^{-1} from LT, VT (above) and the pivot reciprocals;
// ownership as in the factorisation.  X: rows i > k take -l_ik * (row k of X),
// k = 0..NB-1.  Y: with V = U diag(1/u) (unit upper), rows i < q take
// -v_iq * (row q of Y), q = NB-1..0, so Y = V^{-1} and U^{-1} = diag(1/u) Y.
// buf: 4*NB elements of shared scratch.  Writes inv (2 * NB * NB).
template <typename T, int NB, int NT>
__device__ void triangle_inverses(const T *LT, const T *VT, T *buf, const T *rcp, T *inv) {
  static_assert(NB == 64 && NT == 256, "one column pair per lane, 8 rows per warp");
  constexpr int RPW = NB / (NT / 32), TS = diag_tstride<T, NB>();
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int c0 = lane, c1 = NB - 1 - lane, i0 = g * RPW;
  T *rx = buf, *ry = buf + 2 * NB;  // double-buffered row k of X, row q of Y
  T x0[RPW], x1[RPW], y0[RPW], y1[RPW];
#pragma unroll
  for (int t = 0; t < RPW; ++t) {
    x0[t] = y0[t] = (i0 + t == c0) ? T(1) : T(0);
    x1[t] = y1[t] = (i0 + t == c1) ? T(1) : T(0);
  }
  if (threadIdx.x < NB) {
    rx[threadIdx.x] = threadIdx.x == 0 ? T(1) : T(0);
    ry[threadIdx.x] = threadIdx.x == NB - 1 ? T(1) : T(0);
  }
  __syncthreads();
  for (int s = 0; s < NB; ++s) {
    const int b = (s & 1) * NB, nb = NB - b;
    const int k = s, q = NB - 1 - s;
    const T xk0 = rx[b + c0], xk1 = rx[b + c1];
    const T yq0 = ry[b + c0], yq1 = ry[b + c1];
    T l[RPW], v[RPW];
    ld8(LT + k * TS + i0, l);
    ld8(VT + q * TS + i0, v);
#pragma unroll
    for (int t = 0; t < RPW; ++t) {
      x0[t] -= l[t] * xk0;
      x1[t] -= l[t] * xk1;
      y0[t] -= v[t] * yq0;
      y1[t] -= v[t] * yq1;
    }
    if (s + 1 < NB) {
      const int kn = k + 1, qn = q - 1;
      if (kn / RPW == g) {
        rx[nb + c0] = pick(x0, kn - i0);
        rx[nb + c1] = pick(x1, kn - i0);
      }
      if (qn / RPW == g) {
        ry[nb + c0] = pick(y0, qn - i0);
        ry[nb + c1] = pick(y1, qn - i0);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int t = 0; t < RPW; ++t) {
    const int i = i0 + t;
    inv[i * NB + c0] = x0[t];
    inv[i * NB + c1] = x1[t];
    inv[NB * NB + i * NB + c0] = y0[t] * rcp[i];  // rows of U^{-1} take their pivot's reciprocal last
    inv[NB * NB + i * NB + c1] = y1[t] * rcp[i];
  }
}

// ---------------------------------------------------------------------------
// Diagonal block, blocked: the 64 x 64 block as 4 x 4 sub-blocks of 16.  For
// each diagonal sub-block kb: one warp factors it in registers (warp_lu16:
// Doolittle with the EbV column pairs {p, 15-p}, Eq. 6a-c and Eq. 7, pivot
// row and multipliers exchanged by shuffles, no block barrier), two warps
// invert its triangles, then all warps apply 16 x 16 tile products: the L
// blocks below (A_ik U_kk^{-1}), the U blocks right of it (L_kk^{-1} A_kj)
// and the trailing update A_ij -= L_ik U_kj.  The full inverses L11^{-1},
// U11^{-1} then follow block-diagonal by block-diagonal:
//   X_ij = -X_ii sum_{k=j}^{i-1} L_ik X_kj,   Y_ij = -Y_ii sum_{k=i+1}^{j} U_ik Y_kj.
// About twenty barriers in all instead of one per pivot.
// Dynamic shared memory: diagb_smem_bytes<T, NB>().
// ---------------------------------------------------------------------------
constexpr int kSB = 16;  // sub-block order

template <typename T, int NB>
constexpr size_t diagb_smem_bytes() {
  return sizeof(T) * (3 * (size_t)NB * (NB + 1) + 8 * (size_t)kSB * (kSB + 1));
}

// c (this lane's 8 entries of a 16 x 16 tile: row lane/2, columns
// 8*(lane%2) .. +7) +/-= P Q, P and Q 16 x 16 tiles in shared memory.
template <typename T, bool SUB>
__device__ __forceinline__ void wtile_fma(const T *P, int ps, const T *Q, int qs, T (&c)[8]) {
  const int lane = threadIdx.x & 31, r = lane >> 1, cb = (lane & 1) * 8;
#pragma unroll
  for (int k = 0; k < kSB; ++k) {
    const T p = P[r * ps + k];
#pragma unroll
    for (int j = 0; j < 8; ++j) c[j] = SUB ? c[j] - p * Q[k * qs + cb + j] : c[j] + p * Q[k * qs + cb + j];
  }
}
template <typename T>
__device__ __forceinline__ void wtile_get(const T *S, int ss, T (&c)[8]) {
  const int lane = threadIdx.x & 31, r = lane >> 1, cb = (lane & 1) * 8;
#pragma unroll
  for (int j = 0; j < 8; ++j) c[j] = S[r * ss + cb + j];
}
template <typename T>
__device__ __forceinline__ void wtile_put(T *S, int ss, const T (&c)[8]) {
  const int lane = threadIdx.x & 31, r = lane >> 1, cb = (lane & 1) * 8;
#pragma unroll
  for (int j = 0; j < 8; ++j) S[r * ss + cb + j] = c[j];
}

// One warp: Doolittle on the 16 x 16 sub-block at (o, o) of D (row stride
// ld), in place.  Lane (g, p) = (lane / 8, lane % 8) holds rows g, g+4, g+8,
// g+12 of the column pair {p, 15-p}.  rcp[o..o+15] receives the pivot
// reciprocals; the first zero / non-finite pivot below w goes to *bad.
template <typename T>
__device__ __forceinline__ void warp_lu16(T *D, int ld, int o, T *rcp, int w, int *bad) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, p = lane & 7, g = lane >> 3;
  const int c0 = p, c1 = kSB - 1 - p;
  __syncwarp();  // a converged warp: every shuffle below is then a single step
  T v0[4], v1[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    v0[t] = D[(o + g + 4 * t) * ld + o + c0];
    v1[t] = D[(o + g + 4 * t) * ld + o + c1];
  }
  T rc0 = T(0), rc1 = T(0);
  int first_bad = kSB;  // kept in registers: no shared-memory traffic on the pivot chain
#pragma unroll
  for (int r = 0; r < kSB; ++r) {
    const int tr = r >> 2, gr = r & 3;
    const int ps = r < 8 ? r : kSB - 1 - r;  // pair holding column r
    const T pv = __shfl_sync(FULL, r < 8 ? v0[tr] : v1[tr], gr * 8 + ps);
    const T rc = pivot_rcp(pv);
    if (c0 == r) rc0 = rc;
    if (c1 == r) rc1 = rc;
    if (first_bad == kSB && o + r < w && pivot_bad(pv)) first_bad = r;
    if (r == kSB - 1) break;
    T u0 = __shfl_sync(FULL, v0[tr], gr * 8 + p);  // row r, my columns
    T u1 = __shfl_sync(FULL, v1[tr], gr * 8 + p);
    u0 = c0 > r ? u0 : T(0);
    u1 = c1 > r ? u1 : T(0);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      T l = __shfl_sync(FULL, r < 8 ? v0[t] : v1[t], g * 8 + ps) * rc;  // Eq. 6a, my rows
      l = (g + 4 * t > r) ? l : T(0);
      v0[t] -= l * u0;  // Eq. 6c
      v1[t] -= l * u1;
    }
  }
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int i = g + 4 * t;
    D[(o + i) * ld + o + c0] = i > c0 ? v0[t] * rc0 : v0[t];
    D[(o + i) * ld + o + c1] = i > c1 ? v1[t] * rc1 : v1[t];
  }
  if (g == 0) {  // lanes 0..7 hold the reciprocals of the column pairs {p, 15-p}
    rcp[o + c0] = rc0;
    rcp[o + c1] = rc1;
  }
  if (lane == 0 && first_bad < kSB) atomicMin(bad, o + first_bad);
}

// One warp: inverse of the unit lower (lower = true) or upper triangle of the
// factored 16 x 16 sub-block at (o, o) of D, written to the same place of Z.
// Lower: rows i > k take -l_ik (row k).  Upper: rows i < k take
// -(u_ik / u_kk) (row k), k descending, then row i is scaled by 1 / u_ii.
template <typename T, bool LOWER>
__device__ __forceinline__ void warp_tri_inv16(const T *D, T *Z, int ld, int o, const T *rcp) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, p = lane & 7, g = lane >> 3;
  const int c0 = p, c1 = kSB - 1 - p;
  T z0[4], z1[4];
  __syncwarp();  // a converged warp: every shuffle below is then a single step
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    z0[t] = (g + 4 * t == c0) ? T(1) : T(0);
    z1[t] = (g + 4 * t == c1) ? T(1) : T(0);
  }
#pragma unroll
  for (int s = 0; s < kSB; ++s) {
    const int k = LOWER ? s : kSB - 1 - s;
    const int tk = k >> 2, gk = k & 3;
    const T zk0 = __shfl_sync(FULL, z0[tk], gk * 8 + p);  // row k of Z, my columns
    const T zk1 = __shfl_sync(FULL, z1[tk], gk * 8 + p);
    const T rk = rcp[o + k];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int i = g + 4 * t;
      T f = D[(o + i) * ld + o + k];
      f = LOWER ? (i > k ? f : T(0)) : (i < k ? f * rk : T(0));
      z0[t] -= f * zk0;
      z1[t] -= f * zk1;
    }
  }
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int i = g + 4 * t;
    const T sc = LOWER ? T(1) : rcp[o + i];
    Z[(o + i) * ld + o + c0] = z0[t] * sc;
    Z[(o + i) * ld + o + c1] = z1[t] * sc;
  }
}

// One slot row of the register-resident diagonal block's step-k update:
// v[j] -= a w[j] for the columns tx + 16 j > k (live: some row of the warp's
// slot is still active, warp-uniform; rok: this thread's row is).
template <typename T>
__device__ __forceinline__ void lu_slot_update(T (&v)[4], T a, const T (&w)[4], bool live, bool rok, int tx, int k) {
  if (!live) return;
  const int jb = (k + 1) >> 4;  // column blocks j < jb hold no column > k (warp-uniform)
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (j < jb) continue;
    if (rok && tx + 16 * j > k) v[j] -= a * w[j];
  }
}

// Publish pivot row n of the register-resident diagonal block from the warp
// owning it (x: this lane's slot row holding row n or its partner row): the
// FP64 reciprocal of u_nn to rcp[n], the row scaled by it to ws.  The
// half-warp holding row n scales columns tx + 16 j for j < 2, the other half
// (same tx) those for j >= 2, taken by shuffle: two DMUL per lane.
template <typename T>
__device__ __forceinline__ void lu_publish(int n, const T (&x)[4], T *ws, T *rcp, int *bad, int w) {
  const int lane = threadIdx.x & 31, ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  const int nt = n & 15;
  const int src = ((nt & 1) << 4) | nt;  // lane of (n, n)
  T p = x[0];
#pragma unroll
  for (int j = 1; j < 4; ++j)
    if ((n >> 4) == j) p = x[j];
  p = __shfl_sync(0xffffffffu, p, src);
  const T r = pivot_rcp(p);
  const bool mine = ty == nt;  // this half-warp holds row n
  const T y2 = __shfl_xor_sync(0xffffffffu, x[2], 16);
  const T y3 = __shfl_xor_sync(0xffffffffu, x[3], 16);
  const T d0 = (mine ? x[0] : y2) * r;
  const T d1 = (mine ? x[1] : y3) * r;
  ws[tx + (mine ? 0 : 32)] = d0;
  ws[tx + (mine ? 16 : 48)] = d1;
  if (lane == src) {
    rcp[n] = r;
    if (pivot_bad(p) && n < w) atomicMin(bad, n);
  }
}

// The 64 x 64 diagonal block in registers, right-looking Doolittle (Eq.
// 6a-c), one CTA of 256 threads: element (r, c) lives in thread
// (r % 16, c % 16), slot [r / 16][c / 16], so every thread holds rows and
// columns from each quarter of the block and does the same share of every
// step's update (the balance Eq. 7's long/short pairing gives).  A warp owns
// eight whole rows (threads 16 ty .. 16 ty + 15 share a row).
// Step k: a_rc -= a_rk w_kc for r, c > k, with w_kc = u_kc / u_kk the pivot
// row scaled once by its reciprocal (published in shared memory, buffer
// k & 1) and a_rk shuffled inside the owning warp; l_rk = a_rk / u_kk is
// formed for every column at the end.  (An FP64 instruction costs a warp
// slot of the SM's FP64 pipe whatever its active lanes, so the scaling is two
// instructions of one warp per step instead of one per row in every warp.)
// Look-ahead: the warp owning row k+1 updates that row first and publishes
// it before the rest of its update, so the next pivot's chain runs under the
// other warps' updates; one barrier per step.  Rows and columns past w hold
// the identity (and rcp 1).  A zero or non-finite pivot k lowers *bad to k;
// the elimination goes on.  Result: the packed factors to D (shared memory,
// row stride ld, all 64 x 64) when D is set, else to A (the w x w block);
// rcp[k] = 1 / u_kk.  Shared: ws[2][64], rcp[64], *bad (set to 64 here).
template <typename T, bool XV>
__device__ __forceinline__ void diag_lu_regs(MatView<T, XV> A, int64_t k0, int w, T (*ws)[64], T *rcp, int *bad,
                                             T *D, int ld) {
  constexpr int NB = 64;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  const int lane = threadIdx.x & 31;
  T v[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = ty + 16 * i, c = tx + 16 * j;
      v[i][j] = (r < w && c < w) ? A.get(k0 + r, k0 + c) : (r == c ? T(1) : T(0));
    }
  if (threadIdx.x == 0) *bad = NB;
  if (threadIdx.x >= w && threadIdx.x < NB) rcp[threadIdx.x] = T(1);
  __syncthreads();
  const int wrow = ty & ~1;  // this warp's rows: wrow, wrow + 1 (+ 16 i)
  auto slot_row = [&](int i1, T (&x)[4]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      x[j] = v[0][j];
#pragma unroll
      for (int i = 1; i < 4; ++i)
        if (i == i1) x[j] = v[i][j];
    }
  };
  if (wrow == 0) {  // warp 0: row 0
    T x[4];
    slot_row(0, x);
    lu_publish(0, x, ws[0], rcp, bad, w);
  }
  __syncthreads();
  for (int k = 0; k + 1 < w; ++k) {
    const int kt = k & 15, kb = k >> 4, buf = k & 1;
    // a_rk for this thread's rows (the lane of column k in its row shares it)
    T a[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      T s = v[i][0];
#pragma unroll
      for (int j = 1; j < 4; ++j)
        if (kb == j) s = v[i][j];
      a[i] = __shfl_sync(0xffffffffu, s, (lane & 16) | kt);
    }
    T u[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) u[j] = ws[buf][tx + 16 * j];
    const int n1 = k + 1, i1 = n1 >> 4;
    const bool owner = (n1 & 15) >> 1 == (ty >> 1);
    if (owner) {  // row k+1 first, then publish it
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (i == i1) lu_slot_update(v[i], a[i], u, 16 * i + wrow + 1 > k, ty + 16 * i > k, tx, k);
      T x[4];
      slot_row(i1, x);
      lu_publish(n1, x, ws[buf ^ 1], rcp, bad, w);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (!owner || i != i1) lu_slot_update(v[i], a[i], u, 16 * i + wrow + 1 > k, ty + 16 * i > k, tx, k);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = ty + 16 * i, c = tx + 16 * j;
      const T f = c < r ? v[i][j] * rcp[c] : v[i][j];  // l_rc = a_rc / u_cc
      if (D) D[r * ld + c] = f;
      else if (r < w && c < w) A.put(k0 + r, k0 + c, f);
    }
}

// REGS: the elimination by diag_lu_regs (the FP64 default); else the
// blocked one of 16 x 16 sub-blocks below (the binary32 default: measured on
// one 64 x 64 block, FP64 86 us in registers against 119 us blocked, binary32
// 36 us against 18 us).
template <typename T, int NB, int NT, bool XV, bool REGS = (sizeof(T) == 8)>
__device__ __forceinline__ void diag_factor_cta(MatView<T, XV> A, int64_t k0, int w, int32_t *info, T *inv,
                                                unsigned char *dsm) {
  static_assert(NB == 64 && NT == 256, "4 x 4 sub-blocks of 16, 8 warps");
  constexpr int LD = NB + 1, NSB = NB / kSB;
  T *D = reinterpret_cast<T *>(dsm);  // the block, then its packed factors
  T *X = D + NB * LD;                 // L11^{-1}
  T *Y = X + NB * LD;                 // U11^{-1}
  T *scratch = Y + NB * LD;           // one 16 x 17 tile per warp
  __shared__ T rcp[NB];
  __shared__ int bad;
  const int warp = threadIdx.x >> 5;
  T *S = scratch + warp * kSB * (kSB + 1);
  auto blk = [&](T *M, int bi, int bj) { return M + (bi * kSB) * LD + bj * kSB; };
  if constexpr (REGS) {
    // X holds the pivot-row buffers during the elimination
    diag_lu_regs<T, XV>(A, k0, w, reinterpret_cast<T (*)[64]>(X), rcp, &bad, D, LD);
    __syncthreads();
    if (inv) {  // the 16 x 16 diagonal sub-blocks of L11^{-1} (warps 0-3) and U11^{-1} (4-7)
      for (int e = threadIdx.x; e < NB * LD; e += NT) X[e] = Y[e] = T(0);
      __syncthreads();
      if (warp < NSB) warp_tri_inv16<T, true>(D, X, LD, warp * kSB, rcp);
      else warp_tri_inv16<T, false>(D, Y, LD, (warp - NSB) * kSB, rcp);
      __syncthreads();
    }
  } else {
  stage_tile<NB, NT, LD>(D, [&](int i, int j) {
    return (i < w && j < w) ? A.get(k0 + i, k0 + j) : (i == j ? T(1) : T(0));
  });
  for (int e = threadIdx.x; e < NB * LD; e += NT) X[e] = Y[e] = T(0);
  if (threadIdx.x == 0) bad = NB;
  __syncthreads();
  for (int kb = 0; kb < NSB; ++kb) {
    const int o = kb * kSB;
    if (warp == 0) warp_lu16(D, LD, o, rcp, w, &bad);
    __syncthreads();
    if (warp == 0) warp_tri_inv16<T, true>(D, X, LD, o, rcp);
    if (warp == 1) warp_tri_inv16<T, false>(D, Y, LD, o, rcp);
    __syncthreads();
    if (kb + 1 == NSB) break;
    // L blocks below (A_ik U_kk^{-1}) and U blocks right (L_kk^{-1} A_kj), one warp each.
    const int nrest = NSB - 1 - kb;
    if (warp < 2 * nrest) {
      const bool lower = warp < nrest;
      const int m = kb + 1 + (lower ? warp : warp - nrest);
      T c[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) c[j] = T(0);
      if (lower) wtile_fma<T, false>(blk(D, m, kb), LD, blk(Y, kb, kb), LD, c);
      else wtile_fma<T, false>(blk(X, kb, kb), LD, blk(D, kb, m), LD, c);
      __syncwarp();
      wtile_put(lower ? blk(D, m, kb) : blk(D, kb, m), LD, c);
    }
    __syncthreads();
    // Trailing update A_ij -= L_ik U_kj, i, j > kb.
    for (int q = warp; q < nrest * nrest; q += NT / 32) {
      const int bi = kb + 1 + q / nrest, bj = kb + 1 + q % nrest;
      T c[8];
      wtile_get(blk(D, bi, bj), LD, c);
      wtile_fma<T, true>(blk(D, bi, kb), LD, blk(D, kb, bj), LD, c);
      wtile_put(blk(D, bi, bj), LD, c);
    }
    __syncthreads();
  }
  }
  if (threadIdx.x == 0 && bad < NB && info) atomicCAS(info, 0, (int)(k0 + bad + 1));
  for (int e = threadIdx.x; e < NB * NB; e += NT) {
    const int i = e / NB, j = e % NB;
    if (i < w && j < w) A.put(k0 + i, k0 + j, D[i * LD + j]);
  }
  if (!inv) return;
  // Off-diagonal blocks of the inverses, one block distance d at a time.
  for (int d = 1; d < NSB; ++d) {
    const int nb = NSB - d;  // blocks at this distance in each triangle
    if (warp < 2 * nb) {
      const bool lower = warp < nb;
      const int j = lower ? warp : warp - nb;
      T c[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) c[q] = T(0);
      if (lower) {  // X_{j+d, j} = -X_{j+d, j+d} sum_{k=j}^{j+d-1} L_{j+d, k} X_{k, j}
        for (int k = j; k < j + d; ++k) wtile_fma<T, false>(blk(D, j + d, k), LD, blk(X, k, j), LD, c);
      } else {  // Y_{j, j+d} = -Y_{j, j} sum_{k=j+1}^{j+d} U_{j, k} Y_{k, j+d}
        for (int k = j + 1; k <= j + d; ++k) wtile_fma<T, false>(blk(D, j, k), LD, blk(Y, k, j + d), LD, c);
      }
      wtile_put(S, kSB + 1, c);
      __syncwarp();
#pragma unroll
      for (int q = 0; q < 8; ++q) c[q] = T(0);
      if (lower) wtile_fma<T, true>(blk(X, j + d, j + d), LD, S, kSB + 1, c);
      else wtile_fma<T, true>(blk(Y, j, j), LD, S, kSB + 1, c);
      wtile_put(lower ? blk(X, j + d, j) : blk(Y, j, j + d), LD, c);
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < NB * NB; e += NT) {
    const int i = e / NB, j = e % NB;
    inv[e] = X[i * LD + j];
    inv[NB * NB + e] = Y[i * LD + j];
  }
}

// One launch of the diagonal-block factorisation (dynamic shared memory:
// diagb_smem_bytes<T, NB>()).
template <typename T, int NB, int NT, bool XV = false, bool REGS = (sizeof(T) == 8)>
__global__ void __launch_bounds__(NT) k_diag_factor(MatView<T, XV> A, int64_t k0, int w, int32_t *info, T *inv) {
  extern __shared__ __align__(16) unsigned char dsm[];
  diag_factor_cta<T, NB, NT, XV, REGS>(A, k0, w, info, inv, dsm);
}

// The diagonal block alone (no inverses) as its own launch: the FP64 panels
// of the band storages and of small dense systems.  info = k0 + k + 1 for the
// first zero or non-finite pivot k.
template <typename T, bool XV = false>
__global__ void __launch_bounds__(256) k_diag_lu(MatView<T, XV> A, int64_t k0, int w, int32_t *info) {
  __shared__ T ws[2][64];
  __shared__ T rcp[64];
  __shared__ int bad;
  diag_lu_regs<T, XV>(A, k0, w, ws, rcp, &bad, nullptr, 0);
  if (threadIdx.x == 0 && bad < w && info) atomicCAS(info, 0, (int)(k0 + bad + 1));
}


// L21 = A21 U11^{-1} and U12 = L11^{-1} A12 are 64 x 64 x 64 tile products
// against the diagonal-block inverses.  tile_fma: c +/-= P Q for P, Q in
// shared memory (row stride TS, 16-byte rows); thread (ti, tj) accumulates
// rows ti + 16a (a < 4) by the four consecutive columns 4tj .. 4tj+3, so each
// k costs four broadcast loads of P, one vector load of Q and 16 fused
// multiply-adds.  tile_product: Q <- P Q (the result goes back over Q's
// buffer once every thread is done reading).
// Column strips narrower than 64 (CW = 32 or 16) keep the same 256 threads
// on fewer outputs each: rows ti + (1024/CW) a (a < CW/16), columns
// 4tj .. 4tj+3 with tj < CW/4.
template <int CW>
struct StripMap {
  static constexpr int RPT = CW / 16, RS = 1024 / CW, CG = CW / 4;
  static_assert(CW == 64 || CW == 32 || CW == 16, "strip width");
};
// Four consecutive elements (16-byte aligned) of a shared-memory row.
template <typename T>
__device__ __forceinline__ void ld4(const T *p, T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 x = *reinterpret_cast<const float4 *>(p);
    v[0] = x.x, v[1] = x.y, v[2] = x.z, v[3] = x.w;
  } else {
    const double2 x0 = *reinterpret_cast<const double2 *>(p);
    const double2 x1 = *reinterpret_cast<const double2 *>(p + 2);
    v[0] = x0.x, v[1] = x0.y, v[2] = x1.x, v[3] = x1.y;
  }
}
// (Four k at a time: the P row is read with one vector load per four
// multiply-adds of each output; the order of the additions is k = 0, 1, ...)
template <typename T, int NB, int TS, bool SUB, int CW = 64, int QS = TS>  // P rows: stride TS; Q rows: QS
__device__ __forceinline__ void tile_fma(const T *P, const T *Q, T (&c)[StripMap<CW>::RPT][4]) {
  static_assert(NB == 64, "tile mapping assumes 64-row tiles and 256 threads");
  using M = StripMap<CW>;
  const int ti = threadIdx.x / M::CG, tj = threadIdx.x % M::CG;
#pragma unroll 2
  for (int k0 = 0; k0 < NB; k0 += 4) {
    T q[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u) ld4(Q + (k0 + u) * QS + 4 * tj, q[u]);
#pragma unroll
    for (int a = 0; a < M::RPT; ++a) {
      T p[4];
      ld4(P + (ti + M::RS * a) * TS + k0, p);
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int b = 0; b < 4; ++b) c[a][b] = SUB ? c[a][b] - p[u] * q[u][b] : c[a][b] + p[u] * q[u][b];
    }
  }
}
template <typename T, int TS, int CW = 64>
__device__ __forceinline__ void tile_regs(const T *S, T (&c)[StripMap<CW>::RPT][4]) {
  using M = StripMap<CW>;
  const int ti = threadIdx.x / M::CG, tj = threadIdx.x % M::CG;
#pragma unroll
  for (int a = 0; a < M::RPT; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) c[a][b] = S[(ti + M::RS * a) * TS + 4 * tj + b];
}
template <typename T, int TS, int CW = 64>
__device__ __forceinline__ void tile_put(T *S, const T (&c)[StripMap<CW>::RPT][4]) {
  using M = StripMap<CW>;
  const int ti = threadIdx.x / M::CG, tj = threadIdx.x % M::CG;
#pragma unroll
  for (int a = 0; a < M::RPT; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) S[(ti + M::RS * a) * TS + 4 * tj + b] = c[a][b];
}
template <typename T, int NB, int TS, int CW = 64>
__device__ __forceinline__ void tile_product(const T *P, T *Q) {
  T c[StripMap<CW>::RPT][4];
#pragma unroll
  for (int a = 0; a < StripMap<CW>::RPT; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) c[a][b] = T(0);
  tile_fma<T, NB, TS, false, CW>(P, Q, c);
  __syncthreads();
  tile_put<T, TS, CW>(Q, c);
  __syncthreads();
}

// ---------------------------------------------------------------------------
// L21 = A21 U11^{-1}: the L vectors of the block's columns for the rows
// r_begin..r_end-1 below it (Eq. 6a for every row at once).  Without pivoting
// the rows are independent; with U11^{-1} from the diagonal-block kernel each
// 64 x w tile is one small product, computed from shared memory and written
// back coalesced (plus the scaled low-precision shadow of L).
// Dynamic shared memory: pair_smem_bytes<T, NB>().
// ---------------------------------------------------------------------------
template <typename T, typename SH, int NB, bool XV = false>
__global__ void __launch_bounds__(256) k_trsm_ru(MatView<T, XV> A, int64_t k0, int w, int64_t r_begin, int64_t r_end,
                                                 const T *inv, Shadow<SH> sh, Envelope env = {}) {
  static_assert(NB == 64, "tile mapping assumes 64");
  constexpr int TS = diag_tstride<T, NB>();
  extern __shared__ __align__(16) unsigned char dsm[];
  T *At = reinterpret_cast<T *>(dsm);
  T *Ui = At + NB * TS;
  const int64_t r0 = r_begin + (int64_t)blockIdx.x * NB;
  if (env.rows_empty(r0, k0 + w)) return;  // A21 rows zero: L21 rows zero
  const int h = (int)min64(NB, r_end - r0);
  const T *uinv = inv + NB * NB;
  stage_tile<NB, 256, TS>(Ui, [&](int i, int k) { return uinv[i * NB + k]; });
  stage_tile<NB, 256, TS>(At, [&](int i, int k) { return (i < h && k < w) ? A.get(r0 + i, k0 + k) : T(0); });
  __syncthreads();
  tile_product<T, NB, TS>(At, Ui);  // Ui <- At * Ui
  const float s = sh.lb ? sh.scale[0] : 1.f;
  for (int e = threadIdx.x; e < NB * NB; e += 256) {
    const int ii = e / NB, k = e % NB;
    if (ii < h && k < w) {
      const T v = Ui[ii * TS + k];
      A.put(r0 + ii, k0 + k, v);
      if (sh.lb) sh.lb[(r0 + ii) * sh.ld + k0 + k] = from_float<SH>((float)v * s);
    }
  }
}

// The same L21 for RW-row strips (RW = 16 or 32): more CTAs for few rows, for
// the FP64 paths, where one SM's FP64 rate makes a whole 64 x 64 x 64 tile
// product per CTA slow.  Computed transposed, (L21)^T = (U11^{-1})^T A21^T,
// so the strip is the tile product's column strip.
// Dynamic shared memory: pair_smem_bytes<T, NB>().
template <typename T, typename SH, int NB, int RW, bool XV = false>
__global__ void __launch_bounds__(256) k_trsm_ru_strip(MatView<T, XV> A, int64_t k0, int w, int64_t r_begin,
                                                       int64_t r_end, const T *inv, Shadow<SH> sh,
                                                       Envelope env = {}) {
  static_assert(NB == 64, "tile mapping assumes 64");
  constexpr int TS = diag_tstride<T, NB>();
  extern __shared__ __align__(16) unsigned char dsm[];
  T *UiT = reinterpret_cast<T *>(dsm);  // (U11^{-1})^T
  T *AtT = UiT + NB * TS;               // A21 strip transposed: 64 x RW in a 64 x TS buffer
  const int64_t r0 = r_begin + (int64_t)blockIdx.x * RW;
  if (env.rows_empty(r0, k0 + w)) return;  // A21 rows zero: L21 rows zero (RW divides 64)
  const int h = (int)min64(RW, r_end - r0);
  const T *uinv = inv + NB * NB;
  stage_tile<NB, 256, TS>(UiT, [&](int i, int k) { return uinv[k * NB + i]; });
  for (int e = threadIdx.x; e < NB * RW; e += 256) {
    const int i = e / NB, k = e % NB;
    AtT[k * TS + i] = (i < h && k < w) ? A.get(r0 + i, k0 + k) : T(0);
  }
  __syncthreads();
  tile_product<T, NB, TS, RW>(UiT, AtT);  // AtT <- UiT * AtT
  const float s = sh.lb ? sh.scale[0] : 1.f;
  for (int e = threadIdx.x; e < NB * RW; e += 256) {
    const int i = e / NB, k = e % NB;
    if (i < h && k < w) {
      const T v = AtT[k * TS + i];
      A.put(r0 + i, k0 + k, v);
      if (sh.lb) sh.lb[(r0 + i) * sh.ld + k0 + k] = from_float<SH>((float)v * s);
    }
  }
}

// ---------------------------------------------------------------------------
// U12 = L11^{-1} A12: the U vectors of the block's h rows for the columns
// c_begin..c_end-1 (Eq. 6b for every column at once), one h x 64 tile per CTA
// from L11^{-1}.  Also writes the scaled low-precision shadow of U^T.
// Dynamic shared memory: pair_smem_bytes<T, NB>().
// ---------------------------------------------------------------------------
template <typename T, typename SH, int NB, bool XV = false>
__global__ void __launch_bounds__(256) k_trsm_ll(MatView<T, XV> A, int64_t r0, int h, int64_t c_begin, int64_t c_end,
                                                 const T *inv, Shadow<SH> sh, Envelope env = {}) {
  static_assert(NB == 64, "tile mapping assumes 64");
  constexpr int TS = diag_tstride<T, NB>();
  extern __shared__ __align__(16) unsigned char dsm[];
  T *At = reinterpret_cast<T *>(dsm);
  T *Li = At + NB * TS;
  const int64_t c0 = c_begin + (int64_t)blockIdx.x * NB;
  if (env.cols_empty(c0, r0 + h)) return;  // A12 columns zero: U12 columns zero
  const int wc = (int)min64(NB, c_end - c0);
  stage_tile<NB, 256, TS>(Li, [&](int k, int j) { return inv[k * NB + j]; });
  stage_tile<NB, 256, TS>(At, [&](int k, int j) { return (k < h && j < wc) ? A.get(r0 + k, c0 + j) : T(0); });
  __syncthreads();
  tile_product<T, NB, TS>(Li, At);  // At <- Li * At
  for (int e = threadIdx.x; e < NB * NB; e += 256) {
    const int k = e / NB, j = e % NB;
    if (k < h && j < wc) A.put(r0 + k, c0 + j, At[k * TS + j]);
  }
  if (sh.ut) {
    const float s = sh.scale[1];
    for (int e = threadIdx.x; e < NB * NB; e += 256) {
      const int j = e / NB, k = e % NB;
      if (k < h && j < wc) sh.ut[(c0 + j) * sh.ld + r0 + k] = from_float<SH>((float)At[k * TS + j] * s);
    }
  }
}

// ---------------------------------------------------------------------------
// A two-leaf panel's middle step in one launch (recursion nodes of width
// <= 128): U12 = L11^{-1} A12 for the w2 columns right of the left leaf, and
// the trailing update A22 -= L21 U12 of every row below, in the working
// precision.  CTA b owns the 64-row block b of A22; every CTA forms U12 (one
// tile product) from A12.  U12 overwrites A12 in place, so it is stored (with
// its low-precision shadow) by the CTA that arrives last on st->arrive, once
// every CTA has read A12: with more CTAs than fit on the GPU at once, a CTA
// of a later wave would otherwise read U12 where it expects A12.
// Dynamic shared memory: leaf_update_smem_bytes<T, NB>().
// ---------------------------------------------------------------------------
template <typename T, int NB>
constexpr size_t leaf_update_smem_bytes() { return 4 * sizeof(T) * (size_t)NB * diag_tstride<T, NB>(); }

template <typename T, typename SH, int NB>
__global__ void __launch_bounds__(256) k_leaf_update(MatView<T> A, int64_t c0, int w1, int w2, int64_t n,
                                                     const T *inv, Shadow<SH> sh, DevStatus *st) {
  static_assert(NB == 64, "tile mapping assumes 64");
  constexpr int TS = diag_tstride<T, NB>();
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ int last;
  T *Li = reinterpret_cast<T *>(dsm);
  T *U12 = Li + NB * TS;
  T *L21 = U12 + NB * TS;
  T *C = L21 + NB * TS;
  const int64_t cb = c0 + w1;                        // first column (and row) of the right half
  const int64_t r0 = cb + (int64_t)blockIdx.x * NB;  // this CTA's rows of A22
  const int h = (int)min64(NB, n - r0);
  stage_tile<NB, 256, TS>(Li, [&](int i, int k) { return inv[i * NB + k]; });
  stage_tile<NB, 256, TS>(U12, [&](int k, int j) { return (k < w1 && j < w2) ? A.get(c0 + k, cb + j) : T(0); });
  stage_tile<NB, 256, TS>(L21, [&](int i, int k) { return (i < h && k < w1) ? A.get(r0 + i, c0 + k) : T(0); });
  stage_tile<NB, 256, TS>(C, [&](int i, int j) { return (i < h && j < w2) ? A.get(r0 + i, cb + j) : T(0); });
  __syncthreads();
  if (threadIdx.x == 0) {  // A12 is in shared memory: count this CTA as done reading it
    __threadfence();
    last = atomicAdd(&st->arrive, 1) == (int)gridDim.x - 1;
    if (last) st->arrive = 0;  // every CTA has arrived: ready for the next launch
  }
  tile_product<T, NB, TS>(Li, U12);  // U12 = L11^{-1} A12 (Eq. 6b); ends with a barrier
  if (last) {
    for (int e = threadIdx.x; e < NB * NB; e += 256) {
      const int k = e / NB, j = e % NB;
      if (k < w1 && j < w2) A.put(c0 + k, cb + j, U12[k * TS + j]);
    }
    if (sh.ut) {
      const float s = sh.scale[1];
      for (int e = threadIdx.x; e < NB * NB; e += 256) {
        const int j = e / NB, k = e % NB;
        if (k < w1 && j < w2) sh.ut[(cb + j) * sh.ld + c0 + k] = from_float<SH>((float)U12[k * TS + j] * s);
      }
    }
  }
  T acc[4][4];
  tile_regs<T, TS>(C, acc);
  tile_fma<T, NB, TS, true>(L21, U12, acc);  // A22 -= L21 U12 (Eq. 6c, 64 steps aggregated)
  __syncthreads();
  tile_put<T, TS>(C, acc);
  __syncthreads();
  for (int e = threadIdx.x; e < NB * NB; e += 256) {
    const int i = e / NB, j = e % NB;
    if (i < h && j < w2) A.put(r0 + i, cb + j, C[i * TS + j]);
  }
}

// ---------------------------------------------------------------------------
// The left leaf's L21 and the two-leaf middle step in one launch (binary32
// recursion nodes of width <= 128): CTA b owns the 64-row block b below the
// left leaf and forms its L21 block = A21 U11^{-1} (Eq. 6a), writes it (and
// its low-precision shadow), forms U12 = L11^{-1} A12 (Eq. 6b; stored by the
// last CTA to arrive, as in k_leaf_update) and applies A22 -= L21 U12
// (Eq. 6c) from shared memory.  Replaces k_trsm_ru + k_leaf_update: one
// launch and no round trip of L21 through memory on the recursion's
// critical path.  All five input tiles are fetched before any is stored.
// Dynamic shared memory: leaf_ru_update_smem_bytes<T, NB>().
// ---------------------------------------------------------------------------
template <typename T, int NB>
constexpr size_t leaf_ru_update_smem_bytes() { return 5 * sizeof(T) * (size_t)NB * diag_tstride<T, NB>(); }

// After the five tiles are staged (and a barrier): L21 = A21 U11^{-1}, U12 =
// L11^{-1} A12 (stored by the last of the nct CTAs that take part to arrive
// on st->arrive), A22 -= L21 U12; rows r0 .. r0+h of the right half.
template <typename T, typename SH, int NB>
__device__ __forceinline__ void leaf_ru_update_tail(MatView<T> A, int64_t c0, int w1, int w2, int64_t r0, int h,
                                                    Shadow<SH> sh, DevStatus *st, int nct, T *Li, T *U12, T *L21,
                                                    T *At, T *C) {
  constexpr int TS = diag_tstride<T, NB>();
  __shared__ int last;
  const int64_t cb = c0 + w1;
  if (threadIdx.x == 0) {  // A12 is in shared memory: count this CTA as done reading it
    __threadfence();
    last = atomicAdd(&st->arrive, 1) == nct - 1;
    if (last) st->arrive = 0;  // every CTA has arrived: ready for the next launch
  }
  tile_product<T, NB, TS>(At, L21);  // L21 <- A21 U11^{-1}; ends with a barrier
  tile_product<T, NB, TS>(Li, U12);  // U12 = L11^{-1} A12
  {
    const float s = sh.lb ? sh.scale[0] : 1.f;
    for (int e = threadIdx.x; e < NB * NB; e += 256) {
      const int i = e / NB, k = e % NB;
      if (i < h && k < w1) {
        const T v = L21[i * TS + k];
        A.put(r0 + i, c0 + k, v);
        if (sh.lb) sh.lb[(r0 + i) * sh.ld + c0 + k] = from_float<SH>((float)v * s);
      }
    }
  }
  if (last) {
    for (int e = threadIdx.x; e < NB * NB; e += 256) {
      const int k = e / NB, j = e % NB;
      if (k < w1 && j < w2) A.put(c0 + k, cb + j, U12[k * TS + j]);
    }
    if (sh.ut) {
      const float s = sh.scale[1];
      for (int e = threadIdx.x; e < NB * NB; e += 256) {
        const int j = e / NB, k = e % NB;
        if (k < w1 && j < w2) sh.ut[(cb + j) * sh.ld + c0 + k] = from_float<SH>((float)U12[k * TS + j] * s);
      }
    }
  }
  T acc[4][4];
  tile_regs<T, TS>(C, acc);
  tile_fma<T, NB, TS, true>(L21, U12, acc);  // A22 -= L21 U12 (Eq. 6c, 64 steps aggregated)
  __syncthreads();
  tile_put<T, TS>(C, acc);
  __syncthreads();
  for (int e = threadIdx.x; e < NB * NB; e += 256) {
    const int i = e / NB, j = e % NB;
    if (i < h && j < w2) A.put(r0 + i, cb + j, C[i * TS + j]);
  }
}

template <typename T, typename SH, int NB>
__global__ void __launch_bounds__(256) k_leaf_ru_update(MatView<T> A, int64_t c0, int w1, int w2, int64_t n,
                                                        const T *inv, Shadow<SH> sh, DevStatus *st) {
  static_assert(NB == 64, "tile mapping assumes 64");
  constexpr int TS = diag_tstride<T, NB>(), Q = NB * NB / 256;
  extern __shared__ __align__(16) unsigned char dsm[];
  T *Li = reinterpret_cast<T *>(dsm);
  T *U12 = Li + NB * TS;   // A12, then U12
  T *L21 = U12 + NB * TS;  // U11^{-1}, then L21
  T *At = L21 + NB * TS;   // A21
  T *C = At + NB * TS;
  const int64_t cb = c0 + w1;                        // first column (and row) of the right half
  const int64_t r0 = cb + (int64_t)blockIdx.x * NB;  // this CTA's rows
  const int h = (int)min64(NB, n - r0);
  const T *linv = inv, *uinv = inv + NB * NB;
  {
    T f0[Q], f1[Q], f2[Q], f3[Q], f4[Q];
    fetch_tile<NB, 256>(f0, [&](int i, int k) { return linv[i * NB + k]; });
    fetch_tile<NB, 256>(f1, [&](int k, int j) { return (k < w1 && j < w2) ? A.get(c0 + k, cb + j) : T(0); });
    fetch_tile<NB, 256>(f2, [&](int i, int k) { return uinv[i * NB + k]; });
    fetch_tile<NB, 256>(f3, [&](int i, int k) { return (i < h && k < w1) ? A.get(r0 + i, c0 + k) : T(0); });
    fetch_tile<NB, 256>(f4, [&](int i, int j) { return (i < h && j < w2) ? A.get(r0 + i, cb + j) : T(0); });
    put_tile<NB, 256, TS>(Li, f0);
    put_tile<NB, 256, TS>(U12, f1);
    put_tile<NB, 256, TS>(L21, f2);
    put_tile<NB, 256, TS>(At, f3);
    put_tile<NB, 256, TS>(C, f4);
  }
  __syncthreads();
  leaf_ru_update_tail<T, SH, NB>(A, c0, w1, w2, r0, h, sh, st, (int)gridDim.x, Li, U12, L21, At, C);
}

// ---------------------------------------------------------------------------
// A leaf's diagonal block together with the launch that consumes it, as one
// cooperative launch (binary32 recursion).  CTA 0 factors the block (the
// blocked diagonal-block code above) and releases the leaf's flag; every
// other CTA stages its tiles that do not depend on the block, waits for the
// flag (bounded; gives up if the status block reports an error) and then
// applies the block's inverses, read past L1.  This takes the launch gap and
// the consumer's load latency off the recursion's critical path.  All CTAs
// must be co-resident: the host code launches these only when the grid fits.
//   k_diag_l21:        the leaf's L21 for every row below (CTA b >= 1 owns
//                      the 64-row block b-1), as k_trsm_ru;
//   k_diag_l21_update: the left leaf of a two-leaf node with
//                      k_leaf_ru_update's work for the right half.
// Dynamic shared memory: diag_fused_smem_bytes<T, NB>().
// ---------------------------------------------------------------------------
template <typename T, int NB>
constexpr size_t diag_fused_smem_bytes() {
  return diagb_smem_bytes<T, NB>() > leaf_ru_update_smem_bytes<T, NB>() ? diagb_smem_bytes<T, NB>()
                                                                        : leaf_ru_update_smem_bytes<T, NB>();
}

// Thread 0 waits for *flag >= 1; true for every thread once it has.
__device__ __forceinline__ bool cta_wait_flag(const int *flag, DevStatus *st, int where) {
  __shared__ int ok;
  if (threadIdx.x == 0) ok = bounded_wait_geq(flag, 1, st, kSpinLimit, where);
  __syncthreads();
  return ok != 0;
}
__device__ __forceinline__ void cta_release_flag(int *flag) {
  __syncthreads();  // every thread's stores of the block and its inverses are done
  if (threadIdx.x == 0) {
    __threadfence();
    st_release(flag, 1);
  }
}

template <typename T, typename SH, int NB>
__global__ void __launch_bounds__(256) k_diag_l21(MatView<T> A, int64_t c0, int w, int64_t n, int32_t *info, T *inv,
                                                  Shadow<SH> sh, int *flag, DevStatus *st) {
  static_assert(NB == 64, "tile mapping assumes 64");
  constexpr int TS = diag_tstride<T, NB>();
  extern __shared__ __align__(16) unsigned char dsm[];
  if (blockIdx.x == 0) {
    diag_factor_cta<T, NB, 256>(A, c0, w, info, inv, dsm);
    cta_release_flag(flag);
    return;
  }
  T *At = reinterpret_cast<T *>(dsm);
  T *Ui = At + NB * TS;
  const int64_t r0 = c0 + w + (int64_t)(blockIdx.x - 1) * NB;
  const int h = (int)min64(NB, n - r0);
  stage_tile<NB, 256, TS>(At, [&](int i, int k) { return (i < h && k < w) ? A.get(r0 + i, c0 + k) : T(0); });
  if (!cta_wait_flag(flag, st, -1)) return;
  const T *uinv = inv + NB * NB;
  stage_tile<NB, 256, TS>(Ui, [&](int i, int k) { return __ldcg(uinv + i * NB + k); });
  __syncthreads();
  tile_product<T, NB, TS>(At, Ui);  // Ui <- A21 U11^{-1}
  const float s = sh.lb ? sh.scale[0] : 1.f;
  for (int e = threadIdx.x; e < NB * NB; e += 256) {
    const int ii = e / NB, k = e % NB;
    if (ii < h && k < w) {
      const T v = Ui[ii * TS + k];
      A.put(r0 + ii, c0 + k, v);
      if (sh.lb) sh.lb[(r0 + ii) * sh.ld + c0 + k] = from_float<SH>((float)v * s);
    }
  }
}

// k_diag_l21 for the second leaf of a two-leaf node (columns c0+w1 ..
// c0+2*w1, w1 = 64) that also forms the parent node's U12 for the columns
// [cu, cu_end) when nu > 0: CTAs 1 .. nl are the L21 row blocks, CTAs nl+1 ..
// take 16-column strips of U12 = L11^{-1} A12 over the node's two leaves:
// U_0 = L_00^{-1} A_0 and A_1 - L_10 U_0 do not depend on the second
// diagonal block and are formed while CTA 0 factors it; after its flag only
// U_1 = L_11^{-1} (A_1 - L_10 U_0) remains.  c0 here is the node's first
// column; the leaf being factored starts at c0 + 64.
template <typename T, typename SH, int NB>
__global__ void __launch_bounds__(256) k_diag_l21_u12(MatView<T> A, int64_t c0, int w, int64_t n, int nl,
                                                      int64_t cu, int64_t cu_end, int32_t *info, const T *inv0,
                                                      T *inv1, Shadow<SH> sh, int *flag, DevStatus *st) {
  static_assert(NB == 64, "tile mapping assumes 64");
  constexpr int TS = diag_tstride<T, NB>(), CW = 16, Q = NB * NB / 256;
  extern __shared__ __align__(16) unsigned char dsm[];
  const int64_t cl = c0 + NB;  // the leaf factored here
  if (blockIdx.x == 0) {
    diag_factor_cta<T, NB, 256>(A, cl, w, info, inv1, dsm);
    cta_release_flag(flag);
    return;
  }
  if ((int)blockIdx.x <= nl) {  // L21 of the leaf for the 64-row block blockIdx.x - 1 below it
    T *At = reinterpret_cast<T *>(dsm);
    T *Ui = At + NB * TS;
    const int64_t r0 = cl + w + (int64_t)(blockIdx.x - 1) * NB;
    const int h = (int)min64(NB, n - r0);
    stage_tile<NB, 256, TS>(At, [&](int i, int k) { return (i < h && k < w) ? A.get(r0 + i, cl + k) : T(0); });
    if (!cta_wait_flag(flag, st, -5)) return;
    const T *uinv = inv1 + NB * NB;
    stage_tile<NB, 256, TS>(Ui, [&](int i, int k) { return __ldcg(uinv + i * NB + k); });
    __syncthreads();
    tile_product<T, NB, TS>(At, Ui);  // Ui <- A21 U11^{-1}
    const float s = sh.lb ? sh.scale[0] : 1.f;
    for (int e = threadIdx.x; e < NB * NB; e += 256) {
      const int ii = e / NB, k = e % NB;
      if (ii < h && k < w) {
        const T v = Ui[ii * TS + k];
        A.put(r0 + ii, cl + k, v);
        if (sh.lb) sh.lb[(r0 + ii) * sh.ld + cl + k] = from_float<SH>((float)v * s);
      }
    }
    return;
  }
  // U12 strip: columns j0 .. j0+16 of rows c0 .. c0+64+w of the parent node
  T *L0 = reinterpret_cast<T *>(dsm);  // L_00^{-1}, later L_11^{-1}
  T *L10 = L0 + NB * TS;
  T *U0 = L10 + NB * TS;   // 64 x CW strips (row stride TS)
  T *U1 = U0 + NB * TS;
  const int64_t j0 = cu + (int64_t)(blockIdx.x - 1 - nl) * CW;
  const int wc = (int)min64(CW, cu_end - j0);
  {
    T f0[Q], f1[Q];
    fetch_tile<NB, 256>(f0, [&](int i, int k) { return inv0[i * NB + k]; });
    fetch_tile<NB, 256>(f1, [&](int i, int k) { return (i < w) ? A.get(cl + i, c0 + k) : T(0); });
    put_tile<NB, 256, TS>(L0, f0);
    put_tile<NB, 256, TS>(L10, f1);
    for (int e = threadIdx.x; e < NB * CW; e += 256) {
      const int k = e / CW, c = e % CW;
      U0[k * TS + c] = c < wc ? A.get(c0 + k, j0 + c) : T(0);
      U1[k * TS + c] = (k < w && c < wc) ? A.get(cl + k, j0 + c) : T(0);
    }
  }
  __syncthreads();
  tile_product<T, NB, TS, CW>(L0, U0);  // U_0 = L_00^{-1} A_0
  {
    T acc[StripMap<CW>::RPT][4];
    tile_regs<T, TS, CW>(U1, acc);
    tile_fma<T, NB, TS, true, CW>(L10, U0, acc);  // A_1 - L_10 U_0
    __syncthreads();
    tile_put<T, TS, CW>(U1, acc);
  }
  if (!cta_wait_flag(flag, st, -6)) return;
  {
    T f0[Q];
    fetch_tile<NB, 256>(f0, [&](int i, int k) { return __ldcg(inv1 + i * NB + k); });
    put_tile<NB, 256, TS>(L0, f0);  // L_11^{-1}
  }
  __syncthreads();
  tile_product<T, NB, TS, CW>(L0, U1);  // U_1
  const float s = sh.ut ? sh.scale[1] : 1.f;
  for (int e = threadIdx.x; e < 2 * NB * CW; e += 256) {
    const int kk = e / CW, c = e % CW;  // row kk of the node (0 .. 2 NB)
    const int k = kk % NB;
    const T *Ub = kk < NB ? U0 : U1;
    if (c < wc && (kk < NB || k < w)) A.put(c0 + kk, j0 + c, Ub[k * TS + c]);
  }
  if (sh.ut) {
    for (int e = threadIdx.x; e < 2 * NB * CW; e += 256) {
      const int c = e / (2 * NB), kk = e % (2 * NB);
      const int k = kk % NB;
      const T *Ub = kk < NB ? U0 : U1;
      if (c < wc && (kk < NB || k < w)) sh.ut[(j0 + c) * sh.ld + c0 + kk] = from_float<SH>((float)Ub[k * TS + c] * s);
    }
  }
}

template <typename T, typename SH, int NB>
__global__ void __launch_bounds__(256) k_diag_l21_update(MatView<T> A, int64_t c0, int w1, int w2, int64_t n,
                                                         int32_t *info, T *inv, Shadow<SH> sh, int *flag,
                                                         DevStatus *st) {
  static_assert(NB == 64, "tile mapping assumes 64");
  constexpr int TS = diag_tstride<T, NB>(), Q = NB * NB / 256;
  extern __shared__ __align__(16) unsigned char dsm[];
  if (blockIdx.x == 0) {
    diag_factor_cta<T, NB, 256>(A, c0, w1, info, inv, dsm);
    cta_release_flag(flag);
    return;
  }
  T *Li = reinterpret_cast<T *>(dsm);
  T *U12 = Li + NB * TS;
  T *L21 = U12 + NB * TS;
  T *At = L21 + NB * TS;
  T *C = At + NB * TS;
  const int64_t cb = c0 + w1;
  const int64_t r0 = cb + (int64_t)(blockIdx.x - 1) * NB;
  const int h = (int)min64(NB, n - r0);
  {  // the tiles that do not depend on the diagonal block
    T f1[Q], f3[Q], f4[Q];
    fetch_tile<NB, 256>(f1, [&](int k, int j) { return (k < w1 && j < w2) ? A.get(c0 + k, cb + j) : T(0); });
    fetch_tile<NB, 256>(f3, [&](int i, int k) { return (i < h && k < w1) ? A.get(r0 + i, c0 + k) : T(0); });
    fetch_tile<NB, 256>(f4, [&](int i, int j) { return (i < h && j < w2) ? A.get(r0 + i, cb + j) : T(0); });
    put_tile<NB, 256, TS>(U12, f1);
    put_tile<NB, 256, TS>(At, f3);
    put_tile<NB, 256, TS>(C, f4);
  }
  if (!cta_wait_flag(flag, st, -2)) return;
  {
    const T *linv = inv, *uinv = inv + NB * NB;
    T f0[Q], f2[Q];
    fetch_tile<NB, 256>(f0, [&](int i, int k) { return __ldcg(linv + i * NB + k); });
    fetch_tile<NB, 256>(f2, [&](int i, int k) { return __ldcg(uinv + i * NB + k); });
    put_tile<NB, 256, TS>(Li, f0);
    put_tile<NB, 256, TS>(L21, f2);
  }
  __syncthreads();
  leaf_ru_update_tail<T, SH, NB>(A, c0, w1, w2, r0, h, sh, st, (int)gridDim.x - 1, Li, U12, L21, At, C);
}

// ---------------------------------------------------------------------------
// U12 = L11^{-1} A12 for h <= MAXB * NB rows in one launch (Eq. 6b for the
// U vectors of several leaf blocks at once): a left-looking blocked forward
// substitution over the 64-row blocks of L11, one 64-column strip per CTA.
// Block j: acc = A_j - sum_{i<j} L_ji U_i (the finished U_i stay in shared
// memory), U_j = L_jj^{-1} acc through the leaf's inverse; all in the
// working precision.  Replaces the recursive split of small TRSMs (a leaf
// launch and a low-precision GEMM per level) by one launch.  Also writes the
// scaled low-precision shadow of U^T.
// inv: the leaves' inverse slots from row r0 on (slot j, rows r0 + 64 j ..,
// at inv + 2 * NB * NB * j; L^{-1} first).
// Dynamic shared memory: trsm_multi_smem_bytes<T, NB, MAXB>().
// ---------------------------------------------------------------------------
template <typename T, int NB, int MAXB>
constexpr size_t trsm_multi_smem_bytes() { return sizeof(T) * (MAXB + 2) * (size_t)NB * diag_tstride<T, NB>(); }

template <typename T, typename SH, int NB, int MAXB, int CW, bool XV = false>
__global__ void __launch_bounds__(256) k_trsm_ll_multi(MatView<T, XV> A, int64_t r0, int h, int64_t c_begin,
                                                       int64_t c_end, const T *inv, Shadow<SH> sh,
                                                       Envelope env = {}) {
  static_assert(NB == 64, "tile mapping assumes 64");
  constexpr int TS = diag_tstride<T, NB>();
  extern __shared__ __align__(16) unsigned char dsm[];
  T *U = reinterpret_cast<T *>(dsm);  // MAXB finished / current U blocks
  T *Lt = U + MAXB * NB * TS;         // L_ji
  T *Li = Lt + NB * TS;               // L_jj^{-1}
  const int64_t c0 = c_begin + (int64_t)blockIdx.x * CW;
  if (env.cols_empty(c0, r0 + h)) return;  // A12 columns zero: U12 columns zero (CW divides 64)
  const int wc = (int)min64(CW, c_end - c0);
  const int nbk = ceil_div(h, NB);
  // Tile stream, in the order it is consumed: per block j, A_j (this CTA's
  // strip), L_j0 .. L_j,j-1, then L_jj^{-1}.  The next tile's loads are in
  // flight while the current one is being multiplied.
  T pf[NB * NB / 256];
  auto fetch = [&](int j, int pos) {
    const int64_t rj = r0 + (int64_t)j * NB;
    const int hj = min(NB, h - j * NB);
    if (pos == 0) {
      fetch_tile<NB, 256>(pf, [&](int k, int c) { return (k < hj && c < wc) ? A.get(rj + k, c0 + c) : T(0); });
    } else if (pos <= j) {
      const int64_t ri = r0 + (int64_t)(pos - 1) * NB;
      fetch_tile<NB, 256>(pf, [&](int k, int c) { return k < hj ? A.get(rj + k, ri + c) : T(0); });
    } else {
      const T *linv = inv + (int64_t)j * 2 * NB * NB;  // the leaf slot of columns rj..rj+63
      fetch_tile<NB, 256>(pf, [&](int k, int c) { return linv[k * NB + c]; });
    }
  };
  fetch(0, 0);
  for (int j = 0; j < nbk; ++j) {
    const int64_t rj = r0 + (int64_t)j * NB;
    const int hj = min(NB, h - j * NB);
    T *Uj = U + j * NB * TS;
    put_tile<NB, 256, TS>(Uj, pf);
    fetch(j, 1);  // L_j0, or L_jj^{-1} when j == 0
    __syncthreads();
    T acc[StripMap<CW>::RPT][4];
    tile_regs<T, TS, CW>(Uj, acc);
    for (int i = 0; i < j; ++i) {
      __syncthreads();  // the previous product is done with Lt
      put_tile<NB, 256, TS>(Lt, pf);
      fetch(j, i + 2);
      __syncthreads();
      tile_fma<T, NB, TS, true, CW>(Lt, U + i * NB * TS, acc);
    }
    put_tile<NB, 256, TS>(Li, pf);
    if (j + 1 < nbk) fetch(j + 1, 0);
    tile_put<T, TS, CW>(Uj, acc);
    __syncthreads();
    tile_product<T, NB, TS, CW>(Li, Uj);  // U_j = L_jj^{-1} acc
    for (int e = threadIdx.x; e < NB * CW; e += 256) {
      const int k = e / CW, c = e % CW;
      if (k < hj && c < wc) A.put(rj + k, c0 + c, Uj[k * TS + c]);
    }
    if (sh.ut) {
      const float s = sh.scale[1];
      for (int e = threadIdx.x; e < NB * CW; e += 256) {
        const int c = e / NB, k = e % NB;
        if (k < hj && c < wc) sh.ut[(c0 + c) * sh.ld + rj + k] = from_float<SH>((float)Uj[k * TS + c] * s);
      }
    }
  }
}

constexpr int kTrsmMaxBlocks = 4;  // rows of the one-launch TRSM: up to 4 leaves

// The same TRSM with everything resident in shared memory (binary32, strips
// of 16 columns): every tile of L11 it needs -- L_ji (i < j) and the leaf
// inverses L_jj^{-1} -- and the strip of A12 are copied in at once with
// 16-byte cp.async, so the CTA pays one memory latency instead of one per
// tile; then the blocked forward substitution runs from shared memory only.
// Each product sum over K (sum_{i<j} L_ji U_i, then L_jj^{-1} acc) is split
// across four groups of 64 threads, each with a 4 x 4 register block over a
// quarter of K, and reduced through shared memory: a strip this narrow gives
// one thread too few outputs to keep the FMA pipe busy otherwise.
// Requires 16-byte aligned rows (ld % 4 == 0, aligned base); the host code
// falls back to the streaming kernel otherwise.
// Dynamic shared memory: trsm_res_smem_bytes<NB, MAXB>().
constexpr int kResCW = 16, kResUS = kResCW + 4;  // strip width, its row stride
template <int NB, int MAXB>
constexpr size_t trsm_res_smem_bytes() {
  return sizeof(float) * ((size_t)(MAXB * (MAXB + 1) / 2) * NB * diag_tstride<float, NB>() +
                          (size_t)MAXB * NB * kResUS + 4 * (size_t)NB * kResUS);
}

// 16-byte asynchronous copy; `bytes` (0..16) of them are read, the rest zero-filled.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem), "r"(bytes)
               : "memory");
}
// One element's asynchronous copy (4 or 8 bytes, naturally aligned); bytes 0
// zero-fills it.
template <typename T>
__device__ __forceinline__ void cp_async_el(T *smem, const T *gmem, int bytes) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "element size");
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem), "n"((int)sizeof(T)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

template <typename SH, int NB, int MAXB>
__global__ void __launch_bounds__(256) k_trsm_ll_resident(MatView<float> A, int64_t r0, int h, int64_t c_begin,
                                                          int64_t c_end, const float *inv, Shadow<SH> sh) {
  static_assert(NB == 64, "64-row tiles");
  constexpr int TS = diag_tstride<float, NB>(), CW = kResCW, US = kResUS;
  extern __shared__ __align__(16) unsigned char dsm[];
  float *Lbase = reinterpret_cast<float *>(dsm);           // tiles of L11, packed by (j, i)
  float *U = Lbase + (MAXB * (MAXB + 1) / 2) * NB * TS;    // MAXB blocks of 64 x CW
  float *red = U + MAXB * NB * US;                          // 4 partial 64 x CW sums
  auto ltile = [&](int j, int i) { return Lbase + (j * (j + 1) / 2 + i) * NB * TS; };  // i == j: the inverse
  const int nbk = ceil_div(h, NB);
  // One batch of asynchronous copies of L_ji and L_jj^{-1}, kept for every
  // strip this CTA takes (strips s = blockIdx.x + gridDim.x t).
  for (int j = 0; j < nbk; ++j) {
    const int64_t rj = r0 + (int64_t)j * NB;
    const int hj = min(NB, h - j * NB);
    for (int i = 0; i < j; ++i) {
      float *Lt = ltile(j, i);
      const int64_t ri = r0 + (int64_t)i * NB;
      for (int e = threadIdx.x; e < NB * (NB / 4); e += 256) {
        const int k = e / (NB / 4), c = 4 * (e % (NB / 4));
        cp_async16(Lt + k * TS + c, k < hj ? A.base + (rj + k) * A.ld + ri + c : A.base, k < hj ? 16 : 0);
      }
    }
    const float *linv = inv + (int64_t)j * 2 * NB * NB;  // the leaf slot of columns rj..rj+63
    float *Li = ltile(j, j);
    for (int e = threadIdx.x; e < NB * (NB / 4); e += 256) {
      const int k = e / (NB / 4), c = 4 * (e % (NB / 4));
      cp_async16(Li + k * TS + c, linv + k * NB + c, 16);
    }
  }
  const int nstrips = ceil_div(c_end - c_begin, CW);
  for (int strip = blockIdx.x; strip < nstrips; strip += gridDim.x) {
    const int64_t c0 = c_begin + (int64_t)strip * CW;
    const int wc = (int)min64(CW, c_end - c0);
    for (int j = 0; j < nbk; ++j) {  // the strip of A12 (with the L tiles on the first strip)
      const int64_t rj = r0 + (int64_t)j * NB;
      const int hj = min(NB, h - j * NB);
      float *Uj = U + j * NB * US;
      for (int e = threadIdx.x; e < NB * (CW / 4); e += 256) {
        const int k = e / (CW / 4), c = 4 * (e % (CW / 4));
        const int nb = (k < hj) ? 4 * max(0, min(4, wc - c)) : 0;
        cp_async16(Uj + k * US + c, nb ? A.base + (rj + k) * A.ld + c0 + c : A.base, nb);
      }
    }
    cp_async_wait_all();
    __syncthreads();
    // Thread mapping of the split products: group q = tid / 64 takes a quarter
    // of K; inside it thread t holds rows t/4 + 16a (a < 4), columns 4 (t % 4) .. +3.
    const int q = threadIdx.x >> 6, t = threadIdx.x & 63;
    const int pr = t >> 2, pc = 4 * (t & 3);
    // Final mapping: thread tid holds row tid/4, columns 4 (tid % 4) .. +3.
    const int fr = threadIdx.x >> 2, fc = 4 * (threadIdx.x & 3);
    // out = sum over the np products P_m Q_m (P: 64 x 64, stride TS; Q: 64 x CW, stride US).
    auto split_sum = [&](int np, auto P_of, auto Q_of, float (&out)[4]) {
      float c[4][4];
  #pragma unroll
      for (int a = 0; a < 4; ++a)
  #pragma unroll
        for (int b = 0; b < 4; ++b) c[a][b] = 0.f;
      const int kq = 16 * np;  // this group's share of the np * 64 terms
      for (int kk = q * kq; kk < (q + 1) * kq; kk += 16) {
        const float *P = P_of(kk >> 6);
        const float *Q = Q_of(kk >> 6);
        const int k0 = kk & 63;
  #pragma unroll
        for (int k = k0; k < k0 + 16; k += 4) {  // four k per vector load of each P row
          float4 v[4];
  #pragma unroll
          for (int u = 0; u < 4; ++u) v[u] = *reinterpret_cast<const float4 *>(Q + (k + u) * US + pc);
  #pragma unroll
          for (int a = 0; a < 4; ++a) {
            const float4 p4 = *reinterpret_cast<const float4 *>(P + (pr + 16 * a) * TS + k);
            const float p[4] = {p4.x, p4.y, p4.z, p4.w};
  #pragma unroll
            for (int u = 0; u < 4; ++u) {
              c[a][0] += p[u] * v[u].x;
              c[a][1] += p[u] * v[u].y;
              c[a][2] += p[u] * v[u].z;
              c[a][3] += p[u] * v[u].w;
            }
          }
        }
      }
  #pragma unroll
      for (int a = 0; a < 4; ++a)
        *reinterpret_cast<float4 *>(red + q * NB * US + (pr + 16 * a) * US + pc) =
            make_float4(c[a][0], c[a][1], c[a][2], c[a][3]);
      __syncthreads();
  #pragma unroll
      for (int b = 0; b < 4; ++b) out[b] = 0.f;
  #pragma unroll
      for (int g = 0; g < 4; ++g) {
        const float4 v = *reinterpret_cast<const float4 *>(red + g * NB * US + fr * US + fc);
        out[0] += v.x, out[1] += v.y, out[2] += v.z, out[3] += v.w;
      }
      __syncthreads();  // red is free again
    };
    for (int j = 0; j < nbk; ++j) {
      float *Uj = U + j * NB * US;
      float acc[4];
      {
        const float4 v = *reinterpret_cast<const float4 *>(Uj + fr * US + fc);
        acc[0] = v.x, acc[1] = v.y, acc[2] = v.z, acc[3] = v.w;
      }
      if (j > 0) {  // acc = A_j - sum_{i<j} L_ji U_i
        float sum[4];
        split_sum(j, [&](int m) { return (const float *)ltile(j, m); }, [&](int m) { return (const float *)(U + m * NB * US); },
                  sum);
  #pragma unroll
        for (int b = 0; b < 4; ++b) acc[b] -= sum[b];
      }
      *reinterpret_cast<float4 *>(Uj + fr * US + fc) = make_float4(acc[0], acc[1], acc[2], acc[3]);
      __syncthreads();
      float out[4];  // U_j = L_jj^{-1} acc
      split_sum(1, [&](int) { return (const float *)ltile(j, j); }, [&](int) { return (const float *)Uj; }, out);
      *reinterpret_cast<float4 *>(Uj + fr * US + fc) = make_float4(out[0], out[1], out[2], out[3]);
      __syncthreads();
    }
    for (int j = 0; j < nbk; ++j) {
      const int64_t rj = r0 + (int64_t)j * NB;
      const int hj = min(NB, h - j * NB);
      const float *Uj = U + j * NB * US;
      for (int e = threadIdx.x; e < NB * CW; e += 256) {
        const int k = e / CW, c = e % CW;
        if (k < hj && c < wc) A.put(rj + k, c0 + c, Uj[k * US + c]);
      }
      if (sh.ut) {
        const float s = sh.scale[1];
        for (int e = threadIdx.x; e < NB * CW; e += 256) {
          const int c = e / NB, k = e % NB;
          if (k < hj && c < wc) sh.ut[(c0 + c) * sh.ld + rj + k] = from_float<SH>(Uj[k * US + c] * s);
        }
      }
    }
    __syncthreads();  // U and red are rewritten by the next strip
  }
}

// Opt the leaf kernels into more than 48 KB of dynamic shared memory (FP64
// tiles need 66.5 KB); once per process and instantiation.
template <typename T, typename SH>
ebv_status_t prepare_leaf_kernels() {
  static const cudaError_t err = [] {
    const int bytes = (int)pair_smem_bytes<T, kNB>();
    cudaError_t e = set_smem(k_diag_factor<T, kNB, 4 * kNB>, (int)diagb_smem_bytes<T, kNB>());
    if (e == cudaSuccess)
      e = set_smem(k_diag_factor<T, kNB, 4 * kNB, false, !(sizeof(T) == 8)>, (int)diagb_smem_bytes<T, kNB>());
    if (e == cudaSuccess)
      e = set_smem(k_trsm_ru<T, SH, kNB>, bytes);
    if (e == cudaSuccess)
      e = set_smem(k_trsm_ll<T, SH, kNB>, bytes);
    if (e == cudaSuccess)
      e = set_smem(k_trsm_ru_strip<T, SH, kNB, 16>, bytes);
    if (e == cudaSuccess)
      e = set_smem(k_leaf_update<T, SH, kNB>, (int)leaf_update_smem_bytes<T, kNB>());
    if (e == cudaSuccess)
      e = set_smem(k_leaf_ru_update<T, SH, kNB>, (int)leaf_ru_update_smem_bytes<T, kNB>());
    if (e == cudaSuccess)
      e = set_smem(k_diag_l21<T, SH, kNB>, (int)diag_fused_smem_bytes<T, kNB>());
    if (e == cudaSuccess)
      e = set_smem(k_diag_l21_update<T, SH, kNB>, (int)diag_fused_smem_bytes<T, kNB>());
    if (e == cudaSuccess)
      e = set_smem(k_diag_l21_u12<T, SH, kNB>, (int)diag_fused_smem_bytes<T, kNB>());
    const int tb = (int)trsm_multi_smem_bytes<T, kNB, kTrsmMaxBlocks>();
    if (e == cudaSuccess)
      e = set_smem(k_trsm_ll_multi<T, SH, kNB, kTrsmMaxBlocks, 64>, tb);
    if (e == cudaSuccess)
      e = set_smem(k_trsm_ll_multi<T, SH, kNB, kTrsmMaxBlocks, 32>, tb);
    if (e == cudaSuccess)
      e = set_smem(k_trsm_ll_multi<T, SH, kNB, kTrsmMaxBlocks, 16>, tb);
    if constexpr (sizeof(T) == 4) {
      if (e == cudaSuccess)
        e = set_smem(k_trsm_ll_resident<SH, kNB, kTrsmMaxBlocks>, (int)trsm_res_smem_bytes<kNB, kTrsmMaxBlocks>());
    }
    return e;
  }();
  return err == cudaSuccess ? EBV_OK : EBV_ERR_CUDA;
}

// The same opt-in for the kernels the banded factorisation runs through the
// lower-half symmetric and profile views (their own instantiations).
template <typename T>
ebv_status_t prepare_xview_kernels() {
  static const cudaError_t err = [] {
    const int bytes = (int)pair_smem_bytes<T, kNB>();
    cudaError_t e = set_smem(k_diag_factor<T, kNB, 4 * kNB, true>, (int)diagb_smem_bytes<T, kNB>());
    if (e == cudaSuccess)
      e = set_smem(k_diag_factor<T, kNB, 4 * kNB, true, !(sizeof(T) == 8)>, (int)diagb_smem_bytes<T, kNB>());
    if (e == cudaSuccess) e = set_smem(k_trsm_ru<T, float, kNB, true>, bytes);
    if (e == cudaSuccess) e = set_smem(k_trsm_ll<T, float, kNB, true>, bytes);
    if (e == cudaSuccess) e = set_smem(k_trsm_ru_strip<T, float, kNB, 16, true>, bytes);
    if (e == cudaSuccess)
      e = set_smem(k_trsm_ll_multi<T, float, kNB, kTrsmMaxBlocks, 16, true>,
                   (int)trsm_multi_smem_bytes<T, kNB, kTrsmMaxBlocks>());
    return e;
  }();
  return err == cudaSuccess ? EBV_OK : EBV_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// SIMT trailing update in the working precision (Eq. 6c aggregated over K
// steps):  A(m0+i, n0+j) -= sum_k A(m0+i, k0+k) * A(k0+k, n0+j).
// Register-tiled: each thread owns a TM x TN block of C.
// ---------------------------------------------------------------------------
template <typename T, int BM, int BN, int BK, int TM, int TN, bool XV>
__device__ __forceinline__ void gemm_nn_tile(MatView<T, XV> A, int64_t bm, int64_t bn, int64_t mend, int64_t nend,
                                             int64_t k0, int64_t kend, int lower64, Envelope env,
                                             T (*As)[BM + 1], T (*Bs)[BN + 1]) {
  constexpr int NTX = BN / TN, NTY = BM / TM, NT = NTX * NTY;
  const int tx = threadIdx.x % NTX, ty = threadIdx.x / NTX;
  // lower64 (symmetric update): only the tiles of 64-blocks on or below the
  // diagonal (absolute block indices; BM, BN divide 64).
  if (lower64 && bn / 64 > bm / 64) return;
  // outside the envelope (BM, BN divide 64 and m0, n0 start 64-blocks): nothing to subtract
  if (env.rows_empty(bm, kend) || env.cols_empty(bn, kend)) return;
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
      if (gj < nend && A.writable(gi, gj)) {
        T *c = A.at(gi, gj);
        *c = *c - acc[a][b];
      }
    }
  }
}

template <typename T, int BM, int BN, int BK, int TM, int TN, bool XV = false>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    k_gemm_nn(MatView<T, XV> A, int64_t m0, int64_t n0, int64_t k0, int64_t M, int64_t N, int64_t K, int lower64 = 0,
              Envelope env = {}) {
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  gemm_nn_tile<T, BM, BN, BK, TM, TN, XV>(A, m0 + (int64_t)blockIdx.y * BM, n0 + (int64_t)blockIdx.x * BN, m0 + M,
                                          n0 + N, k0, k0 + K, lower64, env, As, Bs);
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
