// Batched factor + solve of many independent small dense systems (project
// addition; the paper factors one matrix at a time) in one persistent launch.
//
// Scheduling follows the pairing idea of Eq. 7, applied across systems: the
// host sorts the systems by cost and lets the cheapest join the most
// expensive while a pair costs no more than the largest system, so work items
// cost about the same; items are ordered by cost and handed out through a
// device counter (CTAs that finish early take the next item).  Each system is
// factored and solved by one CTA in place:
//   per NB-column block: the diagonal block is factored by one warp whose
//   lanes own the column pairs {p, NB-1-p} (equal work per lane over all
//   steps, Eq. 7) and then inverts both triangles; L21 = A21 U11^{-1} and
//   U12 = L11^{-1} A12 are 64-wide tile products; A22 -= L21 U12 runs as
//   register-tiled tiles; then the forward (LY = B) and backward (UX = Y)
//   block substitutions of Eq. 1.
// Variants (per order, from the autotuner): the block width NB (16 or 32;
// 64 too in FP32) and the edge TM of the trailing update's output tiles (32
// or 64; small systems waste less of a 32 x 32 tile).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace ebv {
namespace {

constexpr int BT = 256;              // threads per CTA
constexpr int kMaxBatchOrder = 4096;  // largest order a system may have
constexpr int kMaxBatchRhs = 64;
constexpr int kSchedHeader = 8;
// Variant id v: NB = 16 << (v % 3), TM = 64 >> (v / 3), so 0..2 are NB = 16,
// 32, 64 with 64 x 64 tiles and 3..5 the same with 32 x 32 tiles.  NB = 64
// (ids 2 and 5) is offered in FP32 only: in FP64 its shared memory would
// leave one CTA per SM for every variant.
constexpr int kNumVariants = 6;
constexpr int kVariantShift = 28;
__host__ __device__ constexpr int variant_nb(int v) { return 16 << (v % 3); }
__host__ __device__ constexpr int variant_tm(int v) { return 64 >> (v / 3); }
template <typename T>
constexpr int max_nb() { return sizeof(T) == 4 ? 64 : 32; }
template <typename T>
bool variant_ok(int v) { return v >= 0 && v < kNumVariants && variant_nb(v) <= max_nb<T>(); }

struct BatchArgs {
  const int32_t *n;
  const int32_t *nrhs;
  void *const *a;
  void *const *b;
  const int32_t *sched;
  int32_t *info;
  int *counter;
  DevStatus *st;
};

template <typename T, int NB>
struct BatchSmem {
  T D[NB][NB + 1];   // diagonal block (packed L\U after the warp factorisation)
  T Li[NB][NB + 1];  // L11^{-1}
  T Ui[NB][NB + 1];  // U11^{-1}
  T rcp[NB];         // pivot reciprocals
  T As[NB][64 + 1];  // K-slab of L21 for one 64 x 64 output tile (transposed); also a 64 x NB tile
  T Bs[NB][64 + 1];  // K-slab of U12 for the same tile
  int bad;           // first failing pivot of the system (0-based), or INT32_MAX
};

// Unblocked Doolittle of the w x w block D (w <= NB) by the whole CTA.
// Thread (p, g) owns the column pair {p, NB-1-p} and the rows g, g+NG, ...;
// the pair holds one long and one short column, so all threads do the same
// number of updates over the elimination (Eq. 7).  Multipliers use the pivot
// reciprocal (one division per pivot, thread 0); three barriers per step.
template <typename T, int NB>
__device__ void cta_diag_factor(BatchSmem<T, NB> &sm, int w, int k0) {
  constexpr int NP = NB / 2, NG = BT / NP;
  const int p = threadIdx.x % NP, g = threadIdx.x / NP;
  const int c0 = p, c1 = NB - 1 - p;
  for (int r = 0; r < w; ++r) {
    __syncthreads();  // the block is staged / step r-1's updates are in
    if (threadIdx.x == 0) {
      const T pv = sm.D[r][r];
      sm.rcp[r] = pivot_rcp(pv);
      if (pivot_bad(pv) && sm.bad > k0 + r) sm.bad = k0 + r;
    }
    __syncthreads();
    const T rc = sm.rcp[r];
    for (int i = r + 1 + threadIdx.x; i < w; i += BT) sm.D[i][r] *= rc;  // Eq. 6a
    __syncthreads();
    for (int i = r + 1 + g; i < w; i += NG) {  // Eq. 6c on the owned entries
      const T l = sm.D[i][r];
      if (c0 > r && c0 < w) sm.D[i][c0] -= l * sm.D[r][c0];
      if (c1 > r && c1 < w && c1 != c0) sm.D[i][c1] -= l * sm.D[r][c1];
    }
  }
  __syncthreads();
}

// Inverses of both triangles of the factored block (identity beyond w), one
// warp each: warp 0 builds L11^{-1}, warp 1 U11^{-1}.  A lane owns columns
// c = lane, lane + 32 and substitutes down (L) or up (U) its own column, so
// lanes never wait on one another.
template <typename T, int NB>
__device__ void warp_tri_inverses(BatchSmem<T, NB> &sm, int w, int warp, int lane) {
  if (warp > 1) return;
  T(*Z)[NB + 1] = warp == 0 ? sm.Li : sm.Ui;
  for (int e = lane; e < NB * NB; e += 32) {
    const int i = e / NB, j = e % NB;
    Z[i][j] = (i == j) ? T(1) : T(0);
  }
  __syncwarp();
  for (int c = lane; c < w; c += 32) {
    if (warp == 0) {  // L^{-1}[i][c] = -(l_ic + sum_{c<k<i} l_ik L^{-1}[k][c]), i = c+1 .. w-1
      for (int i = c + 1; i < w; ++i) {
        T s = sm.D[i][c];
        for (int k = c + 1; k < i; ++k) s += sm.D[i][k] * Z[k][c];
        Z[i][c] = -s;
      }
    } else {  // U^{-1}[i][c] = -(sum_{i<k<=c} u_ik U^{-1}[k][c]) / u_ii, i = c .. 0
      Z[c][c] = sm.rcp[c];
      for (int i = c - 1; i >= 0; --i) {
        T s = T(0);
        for (int k = i + 1; k <= c; ++k) s += sm.D[i][k] * Z[k][c];
        Z[i][c] = -s * sm.rcp[i];
      }
    }
  }
  __syncwarp();
}

// Products of an edge tile (it overhangs A22), FP64: only this warp's row
// blocks q < qn (warp-uniform) and the column blocks u < UN (CTA-uniform)
// that hold entries of A22, so no FP64 warp instruction (which costs the
// pipe the same whatever its active lanes) is issued for entries outside it.
template <int TT, int UN, typename T, int NB>
__device__ __forceinline__ void edge_products(const BatchSmem<T, NB> &sm, int ty, int tx, int qn, T (&acc)[TT][TT]) {
#pragma unroll
  for (int q = 0; q < TT; ++q) {
    if (q >= qn) break;
#pragma unroll 4
    for (int k = 0; k < NB; ++k) {
      const T a = sm.As[k][ty + 16 * q];
#pragma unroll
      for (int u = 0; u < UN; ++u) acc[q][u] += a * sm.Bs[k][tx + 16 * u];
    }
  }
}

// A22 -= L21 U12 for the m x m trailing block (rows/cols k0+w..n-1) of one
// system, K = w: TM x TM output tiles (TM = 64: a 4 x 4 register block per
// thread; TM = 32: 2 x 2), taken in row-major order.  The K-slabs of L21 and
// U12 are read with consecutive threads on consecutive addresses of a row
// (coalesced) and stored transposed for L21.  Binary32 is software-pipelined:
// while a tile's products run, the next tile's C and both slabs are already
// loading into registers, so each tile pays no global-memory round trip of
// its own.
template <typename T, int NB, int TM>
__device__ void cta_trailing_update(BatchSmem<T, NB> &sm, T *A, int n, int k0, int w) {
  constexpr int TT = TM / 16;          // outputs per thread along each dimension
  constexpr int SL = NB * TM / BT;     // slab elements per thread (each of L21 and U12)
  static_assert(SL * BT == NB * TM, "slab split");
  const int base = k0 + w, m = n - base;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int nt = (m + TM - 1) / TM, ntiles = nt * nt;
  T cn[TT][TT], an[SL], bn[SL];  // the next tile's C and slabs
  auto fetch = [&](int tile) {
    const int ti = (tile / nt) * TM, tj = (tile % nt) * TM;
#pragma unroll
    for (int q = 0; q < TT; ++q) {
      const int i = ti + ty + 16 * q;
#pragma unroll
      for (int u = 0; u < TT; ++u) {
        const int j = tj + tx + 16 * u;
        cn[q][u] = (i < m && j < m) ? A[(int64_t)(base + i) * n + base + j] : T(0);
      }
    }
#pragma unroll
    for (int v = 0; v < SL; ++v) {
      const int e = threadIdx.x + v * BT;
      const int x = e / NB, k = e % NB;  // L21: row x of the tile, k along the row
      an[v] = (k < w && ti + x < m) ? A[(int64_t)(base + ti + x) * n + k0 + k] : T(0);
      const int kb = e / TM, xb = e % TM;  // U12: row kb, xb along the row
      bn[v] = (kb < w && tj + xb < m) ? A[(int64_t)(k0 + kb) * n + base + tj + xb] : T(0);
    }
  };
  // FP64 (its pipe, not latency, bounds it) fetches each tile when it starts:
  // prefetching too would spill the doubles' registers.
  constexpr bool ahead = sizeof(T) == 4;
  if (ahead && ntiles > 0) fetch(0);
  for (int tile = 0; tile < ntiles; ++tile) {
    if (!ahead) fetch(tile);
    const int ti = (tile / nt) * TM, tj = (tile % nt) * TM;
    T c[TT][TT];
#pragma unroll
    for (int q = 0; q < TT; ++q)
#pragma unroll
      for (int u = 0; u < TT; ++u) c[q][u] = cn[q][u];
#pragma unroll
    for (int v = 0; v < SL; ++v) {
      const int e = threadIdx.x + v * BT;
      sm.As[e % NB][e / NB] = an[v];
      sm.Bs[e / TM][e % TM] = bn[v];
    }
    __syncthreads();
    if (ahead && tile + 1 < ntiles) fetch(tile + 1);  // in flight during the products below
    T acc[TT][TT] = {};
    // (binary32 takes the full-tile loop everywhere: the edge loop's extra
    // shared-memory loads cost it more than the skipped FMAs save)
    if (sizeof(T) == 4 || (ti + TM <= m && tj + TM <= m)) {
#pragma unroll 8
      for (int k = 0; k < NB; ++k) {
        T ra[TT], rb[TT];
#pragma unroll
        for (int q = 0; q < TT; ++q) {
          ra[q] = sm.As[k][ty + 16 * q];
          rb[q] = sm.Bs[k][tx + 16 * q];
        }
#pragma unroll
        for (int q = 0; q < TT; ++q)
#pragma unroll
          for (int u = 0; u < TT; ++u) acc[q][u] += ra[q] * rb[u];
      }
    } else {
      const int qn = min(TT, max(0, (m - ti - (ty & ~1) + 15) / 16));  // this warp's rows: (ty & ~1) + {0, 1}
      const int un = min(TT, (m - tj + 15) / 16);
      if (un == 1) edge_products<TT, 1>(sm, ty, tx, qn, acc);
      if constexpr (TT >= 2)
        if (un == 2) edge_products<TT, 2>(sm, ty, tx, qn, acc);
      if constexpr (TT >= 3)
        if (un == 3) edge_products<TT, 3>(sm, ty, tx, qn, acc);
      if constexpr (TT >= 4)
        if (un == 4) edge_products<TT, 4>(sm, ty, tx, qn, acc);
    }
#pragma unroll
    for (int q = 0; q < TT; ++q) {
      const int i = ti + ty + 16 * q;
      if (i >= m) continue;
      T *row = A + (int64_t)(base + i) * n + base;
#pragma unroll
      for (int u = 0; u < TT; ++u) {
        const int j = tj + tx + 16 * u;
        if (j < m) row[j] = c[q][u] - acc[q][u];
      }
    }
    __syncthreads();
  }
}

// sum_{r < w} f[r] y[r][c] for one row f of a factor (global memory) and a
// solved block y (shared memory): the row's w <= NB entries are loaded
// together (unrolled to NB, predicated), so a row costs one memory round
// trip, not w dependent ones.
template <typename T, int NB>
__device__ __forceinline__ T block_dot(const T *f, int w, const T (*y)[64 + 1], int c) {
  T v[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) v[r] = r < w ? f[r] : T(0);
  T s = T(0);
#pragma unroll
  for (int r = 0; r < NB; ++r)
    if (r < w) s += v[r] * y[r][c];  // rows of y past w are not part of the block
  return s;
}

// In-place LU (packed L\U) of one n x n system, then X = U^{-1} L^{-1} B.
template <typename T, int NB, int TM>
__device__ void cta_lu_solve(BatchSmem<T, NB> &sm, int n, T *A, T *B, int nrhs, int32_t *info) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) sm.bad = INT32_MAX;
  __syncthreads();
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int w = min(NB, n - k0);
    for (int e = threadIdx.x; e < NB * NB; e += BT) {
      const int i = e / NB, j = e % NB;
      sm.D[i][j] = (i < w && j < w) ? A[(int64_t)(k0 + i) * n + k0 + j] : (i == j ? T(1) : T(0));
    }
    __syncthreads();
    cta_diag_factor<T, NB>(sm, w, k0);
    warp_tri_inverses<T, NB>(sm, w, warp, lane);
    __syncthreads();
    for (int e = threadIdx.x; e < w * w; e += BT) {
      const int i = e / w, j = e % w;
      A[(int64_t)(k0 + i) * n + k0 + j] = sm.D[i][j];
    }
    // L21 = A21 U11^{-1} (Eq. 6a for every row below), 64-row tiles, the
    // next tile's entries loading into registers while one is multiplied.
    constexpr int PT = 64 * NB / BT;  // tile entries per thread
    T pf[PT];
    auto fetch_l = [&](int t0) {
      const int h = min(64, n - t0);
#pragma unroll
      for (int v = 0; v < PT; ++v) {
        const int e = threadIdx.x + v * BT, r = e / NB, k = e % NB;
        pf[v] = (r < h && k < w) ? A[(int64_t)(t0 + r) * n + k0 + k] : T(0);
      }
    };
    T(*tile)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(&sm.As[0][0]);  // 64 x NB fits in As + Bs
    if (k0 + w < n) fetch_l(k0 + w);
    for (int t0 = k0 + w; t0 < n; t0 += 64) {
      const int h = min(64, n - t0);
      __syncthreads();
#pragma unroll
      for (int v = 0; v < PT; ++v) {
        const int e = threadIdx.x + v * BT;
        tile[e / NB][e % NB] = pf[v];
      }
      __syncthreads();
      if (t0 + 64 < n) fetch_l(t0 + 64);
      const int r = threadIdx.x >> 2, cq = threadIdx.x & 3;
      T out[NB / 4];
#pragma unroll
      for (int q = 0; q < NB / 4; ++q) out[q] = T(0);
#pragma unroll 4
      for (int k = 0; k < NB; ++k) {
        const T a = tile[r][k];
#pragma unroll
        for (int q = 0; q < NB / 4; ++q) out[q] += a * sm.Ui[k][cq + 4 * q];
      }
      if (r < h)
#pragma unroll
        for (int q = 0; q < NB / 4; ++q)
          if (cq + 4 * q < w) A[(int64_t)(t0 + r) * n + k0 + cq + 4 * q] = out[q];
    }
    // U12 = L11^{-1} A12 (Eq. 6b for every column to the right), 64-column
    // tiles, prefetched the same way.
    auto fetch_u = [&](int t0) {
      const int h = min(64, n - t0);
#pragma unroll
      for (int v = 0; v < PT; ++v) {
        const int e = threadIdx.x + v * BT, k = e / 64, c = e % 64;
        pf[v] = (k < w && c < h) ? A[(int64_t)(k0 + k) * n + t0 + c] : T(0);
      }
    };
    if (k0 + w < n) fetch_u(k0 + w);
    for (int t0 = k0 + w; t0 < n; t0 += 64) {
      const int h = min(64, n - t0);
      __syncthreads();
#pragma unroll
      for (int v = 0; v < PT; ++v) {
        const int e = threadIdx.x + v * BT;
        sm.Bs[e / 64][e % 64] = pf[v];
      }
      __syncthreads();
      if (t0 + 64 < n) fetch_u(t0 + 64);
      const int c = threadIdx.x & 63, rg = threadIdx.x >> 6;
      T out[NB / 4];
#pragma unroll
      for (int q = 0; q < NB / 4; ++q) out[q] = T(0);
#pragma unroll 4
      for (int k = 0; k < NB; ++k) {
        const T b = sm.Bs[k][c];
#pragma unroll
        for (int q = 0; q < NB / 4; ++q) out[q] += sm.Li[rg + 4 * q][k] * b;
      }
      if (c < h)
#pragma unroll
        for (int q = 0; q < NB / 4; ++q)
          if (rg + 4 * q < w) A[(int64_t)(k0 + rg + 4 * q) * n + t0 + c] = out[q];
    }
    __syncthreads();
    if (n - k0 - w > 0) cta_trailing_update<T, NB, TM>(sm, A, n, k0, w);
    __syncthreads();
  }
  if (threadIdx.x == 0) *info = sm.bad == INT32_MAX ? 0 : sm.bad + 1;
  if (nrhs <= 0) return;
  // Forward substitution LY = B (unit lower), block by block (Eq. 1): the
  // diagonal block of L and the block's right-hand-side rows in shared
  // memory (the factorisation is done with D and As), warp 0 solving the
  // block there; then every later row takes the block's contribution,
  // accumulated from zero and subtracted once.
  T(*Ts)[NB + 1] = sm.D;
  T(*Bs)[64 + 1] = sm.As;  // NB x nrhs (nrhs <= 64)
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int w = min(NB, n - k0);
    for (int e = threadIdx.x; e < w * w; e += BT) {
      const int i = e / w, j = e % w;
      Ts[i][j] = j < i ? A[(int64_t)(k0 + i) * n + k0 + j] : T(0);
    }
    for (int e = threadIdx.x; e < w * nrhs; e += BT) Bs[e / nrhs][e % nrhs] = B[(int64_t)k0 * nrhs + e];
    __syncthreads();
    if (warp == 0) {
      for (int r = 0; r < w; ++r) {
        for (int e = lane; e < (w - 1 - r) * nrhs; e += 32) {
          const int i = r + 1 + e / nrhs, c = e % nrhs;
          Bs[i][c] -= Ts[i][r] * Bs[r][c];
        }
        __syncwarp();
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < w * nrhs; e += BT) B[(int64_t)k0 * nrhs + e] = Bs[e / nrhs][e % nrhs];
    for (int e = threadIdx.x; e < (n - k0 - w) * nrhs; e += BT) {
      const int i = k0 + w + e / nrhs, c = e % nrhs;
      B[(int64_t)i * nrhs + c] -= block_dot<T, NB>(A + (int64_t)i * n + k0, w, Bs, c);
    }
    __syncthreads();
  }
  // Backward substitution UX = Y, diagonal through pivot reciprocals, the
  // same way from the last block up.
  for (int kend = n; kend > 0; kend -= NB) {
    const int k0 = max(0, kend - NB), w = kend - k0;
    for (int e = threadIdx.x; e < w * w; e += BT) {
      const int i = e / w, j = e % w;
      Ts[i][j] = j >= i ? A[(int64_t)(k0 + i) * n + k0 + j] : T(0);
    }
    for (int e = threadIdx.x; e < w * nrhs; e += BT) Bs[e / nrhs][e % nrhs] = B[(int64_t)k0 * nrhs + e];
    __syncthreads();
    if (warp == 0) {
      for (int r = w - 1; r >= 0; --r) {
        const T rc = pivot_rcp(Ts[r][r]);
        for (int c = lane; c < nrhs; c += 32) Bs[r][c] *= rc;
        __syncwarp();
        for (int e = lane; e < r * nrhs; e += 32) {
          const int i = e / nrhs, c = e % nrhs;
          Bs[i][c] -= Ts[i][r] * Bs[r][c];
        }
        __syncwarp();
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < w * nrhs; e += BT) B[(int64_t)k0 * nrhs + e] = Bs[e / nrhs][e % nrhs];
    for (int e = threadIdx.x; e < k0 * nrhs; e += BT) {
      const int i = e / nrhs, c = e % nrhs;
      B[(int64_t)i * nrhs + c] -= block_dot<T, NB>(A + (int64_t)i * n + k0, w, Bs, c);
    }
    __syncthreads();
  }
}

// Persistent kernel: each CTA takes (long, short) pairs from the schedule
// through a device counter until none is left.
template <typename T>
__global__ void __launch_bounds__(BT, 2) k_batched(BatchArgs args) {
  extern __shared__ __align__(16) unsigned char smraw[];  // sizeof(BatchSmem<T, max_nb<T>()>)
  __shared__ int s_item;
  const int P = args.sched[0];
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(args.counter, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= P) break;
    for (int h = 0; h < 2; ++h) {
      const int code = args.sched[kSchedHeader + 2 * item + h];
      if (code < 0) continue;
      const int sys = code & ((1 << kVariantShift) - 1), variant = code >> kVariantShift;
      const int n = args.n[sys], nrhs = args.nrhs[sys];
      if (n < 0 || n > kMaxBatchOrder || nrhs < 0 || nrhs > kMaxBatchRhs) {
        if (threadIdx.x == 0) args.info[sys] = -1;  // rejected: outside the supported sizes
        continue;
      }
      T *A = (T *)args.a[sys];
      T *B = (T *)args.b[sys];
      switch (variant) {
        case 0: cta_lu_solve<T, 16, 64>(*reinterpret_cast<BatchSmem<T, 16> *>(smraw), n, A, B, nrhs, &args.info[sys]); break;
        case 3: cta_lu_solve<T, 16, 32>(*reinterpret_cast<BatchSmem<T, 16> *>(smraw), n, A, B, nrhs, &args.info[sys]); break;
        case 4: cta_lu_solve<T, 32, 32>(*reinterpret_cast<BatchSmem<T, 32> *>(smraw), n, A, B, nrhs, &args.info[sys]); break;
        case 2:
        case 5:
          if constexpr (max_nb<T>() >= 64) {
            if (variant == 2)
              cta_lu_solve<T, 64, 64>(*reinterpret_cast<BatchSmem<T, 64> *>(smraw), n, A, B, nrhs, &args.info[sys]);
            else
              cta_lu_solve<T, 64, 32>(*reinterpret_cast<BatchSmem<T, 64> *>(smraw), n, A, B, nrhs, &args.info[sys]);
            break;
          }
          [[fallthrough]];
        default: cta_lu_solve<T, 32, 64>(*reinterpret_cast<BatchSmem<T, 32> *>(smraw), n, A, B, nrhs, &args.info[sys]); break;
      }
      __syncthreads();
    }
  }
}

int default_variant(int n) { return n <= 64 ? 0 : 1; }

// CTAs of the persistent launch that fit on the device at once (0 on error).
template <typename T>
int resident_ctas() {
  static const int r = [] {
    constexpr int smem = (int)sizeof(BatchSmem<T, max_nb<T>()>);
    if (set_smem(k_batched<T>, smem) != cudaSuccess)
      return 0;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batched<T>, BT, smem);
    return sms * per_sm;
  }();
  return r;
}

template <typename T>
ebv_status_t launch_batched(const BatchArgs &args, int items, cudaStream_t s) {
  if (items <= 0) return EBV_OK;
  const int resident = resident_ctas<T>();
  if (resident <= 0) return EBV_ERR_CUDA;
  const int grid = std::min(items, resident);
  prof::Scope ps(s, prof::kBatched, 0.0);
  k_batched<T><<<grid, BT, sizeof(BatchSmem<T, max_nb<T>()>), s>>>(args);
  return launch_ok();
}

// Diagonally dominant test matrices for the autotuner: a_ii = 1, a_ij a
// hash-based uniform in [-0.5, 0.5] / (n - 1); b = 1.
template <typename T>
__global__ void k_fill_dd(T *a, T *b, int n, int reps) {
  const int64_t total = (int64_t)reps * n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ij = e % ((int64_t)n * n);
    const int i = (int)(ij / n), j = (int)(ij % n);
    uint32_t h = (uint32_t)(e * 2654435761u) ^ 0x9E3779B9u;
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    const float u = (h >> 8) * (1.0f / 16777216.0f) - 0.5f;
    a[e] = (i == j) ? T(1) : (T)(u / (float)max(1, n - 1));
    if (j == 0) b[e / n] = T(1);
  }
}

// Work items of a batch: Eq. 7's equalisation applied across systems.  The
// systems are sorted by cost (2n^3/3 + 2n^2 nrhs flops, + 1 so that empty
// systems still count); walking from the most expensive system down and from
// the cheapest up, a short system joins a long one while the pair costs no
// more than the single most expensive system, the time every CTA's work is
// equalised towards.  Items come out in decreasing cost (stable: equal costs
// keep the systems' order).  EBV_ERR_ARG for an order outside 0..4096 or a
// right-hand-side count outside 0..64.
struct Item {
  double cost;
  int32_t sys[2];  // the long system, and the short one or -1
};

ebv_status_t pair_systems(int64_t batch, const int32_t *n_host, const int32_t *nrhs_host, std::vector<Item> &items) {
  if (batch > 0 && (!n_host || !nrhs_host)) return EBV_ERR_ARG;
  std::vector<double> cost((size_t)batch);
  for (int64_t s = 0; s < batch; ++s) {
    const int n = n_host[s], r = nrhs_host[s];
    if (n < 0 || n > kMaxBatchOrder || r < 0 || r > kMaxBatchRhs) return EBV_ERR_ARG;
    cost[s] = 2.0 * n * n * n / 3.0 + 2.0 * n * n * r + 1.0;
  }
  std::vector<int32_t> order((size_t)batch);
  for (int64_t s = 0; s < batch; ++s) order[s] = (int32_t)s;
  std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return cost[x] > cost[y]; });
  items.clear();
  items.reserve((size_t)batch);
  const double cap = batch > 0 ? cost[order[0]] : 0.0;
  for (int64_t i = 0, j = batch - 1; i <= j; ++i) {
    const int32_t lo = order[i];
    if (j > i && cost[lo] + cost[order[j]] <= cap) {
      const int32_t sh = order[j--];
      items.push_back({cost[lo] + cost[sh], {lo, sh}});
    } else {
      items.push_back({cost[lo], {lo, -1}});
    }
  }
  std::stable_sort(items.begin(), items.end(), [](const Item &x, const Item &y) { return x.cost > y.cost; });
  return EBV_OK;
}

}  // namespace
}  // namespace ebv

using namespace ebv;

extern "C" {

int64_t ebv_batch_schedule_len(int64_t batch) { return batch < 0 ? 0 : 2 * batch + kSchedHeader; }

size_t ebv_batch_workspace_size(int64_t) { return kStatusBytes; }

ebv_status_t ebv_batch_schedule(int64_t batch, const int32_t *n_host, const int32_t *nrhs_host,
                                const int8_t *variant_of_n, int32_t *schedule_host) {
  if (batch < 0 || batch >= (int64_t(1) << kVariantShift) || !schedule_host) return EBV_ERR_ARG;
  std::vector<Item> items;
  EBV_TRY(pair_systems(batch, n_host, nrhs_host, items));
  auto code = [&](int32_t s) -> int32_t {
    if (s < 0) return -1;
    const int n = n_host[s];
    int v = default_variant(n);
    if (variant_of_n && n >= 1 && variant_of_n[n - 1] >= 0 && variant_of_n[n - 1] < kNumVariants)
      v = variant_of_n[n - 1];
    return s | (v << kVariantShift);
  };
  const int64_t P = (int64_t)items.size();
  std::memset(schedule_host, 0, sizeof(int32_t) * (size_t)ebv_batch_schedule_len(batch));
  schedule_host[0] = (int32_t)P;
  schedule_host[1] = (int32_t)batch;
  for (int64_t p = 0; p < P; ++p) {
    schedule_host[kSchedHeader + 2 * p] = code(items[p].sys[0]);
    schedule_host[kSchedHeader + 2 * p + 1] = code(items[p].sys[1]);
  }
  return EBV_OK;
}

ebv_status_t ebv_batch_partition(int64_t batch, const int32_t *n_host, const int32_t *nrhs_host, int32_t nranks,
                                 int32_t *rank_of_host, double *cost_of_rank_host) {
  if (batch < 0 || batch >= (int64_t(1) << kVariantShift) || nranks < 1 || nranks > 65536) return EBV_ERR_ARG;
  if (batch > 0 && !rank_of_host) return EBV_ERR_ARG;
  std::vector<Item> items;
  EBV_TRY(pair_systems(batch, n_host, nrhs_host, items));
  // Longest processing time first: the items (long/short pairs, already in
  // decreasing cost) go one by one to the rank with the least work so far,
  // the lowest rank on ties.  No rank then ends more than one item's cost
  // above the average.
  std::vector<double> load((size_t)nranks, 0.0);
  for (const Item &it : items) {
    int32_t r = 0;
    for (int32_t q = 1; q < nranks; ++q)
      if (load[q] < load[r]) r = q;
    load[r] += it.cost;
    for (int h = 0; h < 2; ++h)
      if (it.sys[h] >= 0) rank_of_host[it.sys[h]] = r;
  }
  if (cost_of_rank_host)
    for (int32_t q = 0; q < nranks; ++q) cost_of_rank_host[q] = load[q];
  return EBV_OK;
}

ebv_status_t ebv_factor_solve_batched(int64_t batch, const int32_t *n_dev, const int32_t *nrhs_dev,
                                      void *const *a_ptrs_dev, void *const *b_ptrs_dev, ebv_prec_t prec,
                                      const int32_t *schedule_dev, int32_t *info_dev, void *ws, size_t ws_bytes,
                                      ebv_stream_t stream) {
  if (batch < 0 || batch >= (int64_t(1) << kVariantShift)) return EBV_ERR_ARG;
  if (prec != EBV_FP64 && prec != EBV_FP32) return EBV_ERR_ARG;
  if (batch == 0) return EBV_OK;
  if (!n_dev || !nrhs_dev || !a_ptrs_dev || !b_ptrs_dev || !schedule_dev || !info_dev) return EBV_ERR_ARG;
  if (!ws || ((uintptr_t)ws % 256) != 0 || ws_bytes < kStatusBytes) return EBV_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  EBV_CU(cudaMemsetAsync(ws, 0, kStatusBytes, s));
  BatchArgs args{n_dev, nrhs_dev, a_ptrs_dev, b_ptrs_dev, schedule_dev, info_dev, (int *)((char *)ws + 64),
                 (DevStatus *)ws};
  const int items = (int)batch;  // upper bound on the schedule's work items (the kernel reads their count)
  return prec == EBV_FP64 ? launch_batched<double>(args, items, s) : launch_batched<float>(args, items, s);
}

// Scratch layout of the autotuner for `reps` systems of order <= max_n:
// matrices, right-hand sides, pointer arrays, order/rhs arrays, info,
// schedule, status block.
size_t ebv_batch_autotune_scratch(int32_t max_n, int32_t reps, ebv_prec_t prec) {
  if (max_n < 1 || max_n > kMaxBatchOrder || reps < 1 || (prec != EBV_FP64 && prec != EBV_FP32)) return 0;
  const size_t ts = prec == EBV_FP64 ? 8 : 4;
  size_t off = kStatusBytes;
  off = align256(off + (size_t)reps * max_n * max_n * ts);
  off = align256(off + (size_t)reps * max_n * ts);
  off = align256(off + 2 * (size_t)reps * sizeof(void *));
  off = align256(off + 3 * (size_t)reps * sizeof(int32_t));
  off = align256(off + sizeof(int32_t) * (size_t)ebv_batch_schedule_len(reps));
  return off;
}

ebv_status_t ebv_batch_autotune(const int32_t *orders, int32_t count, int32_t reps, ebv_prec_t prec, void *scratch_dev,
                                size_t scratch_bytes, int8_t *best_variant_host, float *ms_host, ebv_stream_t stream) {
  if (!orders || count < 1 || reps < 1 || !best_variant_host) return EBV_ERR_ARG;
  if (prec != EBV_FP64 && prec != EBV_FP32) return EBV_ERR_ARG;
  int max_n = 0;
  for (int i = 0; i < count; ++i) {
    if (orders[i] < 1 || orders[i] > kMaxBatchOrder) return EBV_ERR_ARG;
    max_n = std::max(max_n, (int)orders[i]);
  }
  const size_t need = ebv_batch_autotune_scratch(max_n, reps, prec);
  if (!scratch_dev || scratch_bytes < need || ((uintptr_t)scratch_dev % 256) != 0) return EBV_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t ts = prec == EBV_FP64 ? 8 : 4;
  char *base = (char *)scratch_dev;
  size_t off = kStatusBytes;
  char *amat = base + off;
  off = align256(off + (size_t)reps * max_n * max_n * ts);
  char *bvec = base + off;
  off = align256(off + (size_t)reps * max_n * ts);
  void **ptrs = (void **)(base + off);
  off = align256(off + 2 * (size_t)reps * sizeof(void *));
  int32_t *ints = (int32_t *)(base + off);
  off = align256(off + 3 * (size_t)reps * sizeof(int32_t));
  int32_t *sched = (int32_t *)(base + off);
  std::vector<void *> hp(2 * (size_t)reps);
  std::vector<int32_t> hn(reps), hr(reps, 1), hs((size_t)ebv_batch_schedule_len(reps));
  std::vector<int8_t> vmap(kMaxBatchOrder);
  cudaEvent_t e0, e1;
  EBV_CU(cudaEventCreate(&e0));
  EBV_CU(cudaEventCreate(&e1));
  ebv_status_t status = EBV_OK;
  for (int oi = 0; oi < count && status == EBV_OK; ++oi) {
    const int n = orders[oi];
    for (int r = 0; r < reps; ++r) {
      hp[r] = amat + (size_t)r * n * n * ts;
      hp[reps + r] = bvec + (size_t)r * n * ts;
      hn[r] = n;
    }
    if (cudaMemcpyAsync(ptrs, hp.data(), hp.size() * sizeof(void *), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(ints, hn.data(), reps * sizeof(int32_t), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(ints + reps, hr.data(), reps * sizeof(int32_t), cudaMemcpyHostToDevice, s) != cudaSuccess) {
      status = EBV_ERR_CUDA;
      break;
    }
    float best = 0.f;
    int bestv = default_variant(n);
    bool have = false;
    for (int v = 0; v < kNumVariants; ++v) {
      if (!(prec == EBV_FP64 ? variant_ok<double>(v) : variant_ok<float>(v))) {
        if (ms_host) ms_host[oi * kNumVariants + v] = -1.f;  // not offered in this precision
        continue;
      }
      std::fill(vmap.begin(), vmap.end(), (int8_t)v);
      ebv_batch_schedule(reps, hn.data(), hr.data(), vmap.data(), hs.data());
      cudaMemcpyAsync(sched, hs.data(), hs.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
      const int grid = std::max(1, std::min((int)((int64_t)reps * n * n / 65536) + 1, 4096));
      float tms = 1e30f;
      for (int trial = 0; trial < 2; ++trial) {  // the first run warms up
        if (prec == EBV_FP64)
          k_fill_dd<double><<<grid, 256, 0, s>>>((double *)amat, (double *)bvec, n, reps);
        else
          k_fill_dd<float><<<grid, 256, 0, s>>>((float *)amat, (float *)bvec, n, reps);
        cudaEventRecord(e0, s);
        status = ebv_factor_solve_batched(reps, ints, ints + reps, ptrs, ptrs + reps, prec, sched, ints + 2 * reps,
                                          base, kStatusBytes, stream);
        cudaEventRecord(e1, s);
        if (status != EBV_OK || cudaEventSynchronize(e1) != cudaSuccess) {
          if (status == EBV_OK) status = EBV_ERR_CUDA;
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (trial > 0) tms = ms;
      }
      if (status != EBV_OK) break;
      if (ms_host) ms_host[oi * kNumVariants + v] = tms;
      if (!have || tms < best) {
        best = tms;
        bestv = v;
        have = true;
      }
    }
    best_variant_host[oi] = (int8_t)bestv;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return status;
}

}  // extern "C"
