// Triangular solves (Eq. 1: LY = B, then UX = Y) and iterative-refinement
// kernels.
#pragma once

#include "dense_kernels.cuh"
#include "multiword.cuh"

namespace ebv {
namespace {  // internal linkage: every translation unit gets its own kernels

// ---------------------------------------------------------------------------
// Per diagonal block b of the packed factors, at dinv + b * 4 * NB * NB:
// L_bb^{-1}, U_bb^{-1}, L_bb^{-1} L_b,b-1 and U_bb^{-1} U_b,b+1 (zero where
// the neighbour block does not exist).  One CTA per block.  The inverses make
// each diagonal solve of the substitution a tile product; the coupling
// products let a substitution step fold its predecessor and solve in one
// product: x_b = L_bb^{-1} acc - (L_bb^{-1} L_b,b-1) x_{b-1}.
// Dynamic shared memory: diag_smem_bytes<T, NB>().
// ---------------------------------------------------------------------------
template <typename T, int NB, bool XV = false>
__global__ void __launch_bounds__(4 * NB) k_diag_inverses(MatView<T, XV> F, int64_t n, T *dinv) {
  extern __shared__ __align__(16) unsigned char dsm[];
  T(*D)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(dsm);
  T *LT = reinterpret_cast<T *>(dsm + sizeof(T) * NB * (NB + 1));
  T *VT = LT + NB * diag_tstride<T, NB>();
  T *buf = VT + NB * diag_tstride<T, NB>();
  __shared__ T rcp[NB];
  const int64_t i0 = (int64_t)blockIdx.x * NB;
  const int hb = (int)min64(NB, n - i0);
  stage_tile<NB, 4 * NB, NB + 1>(&D[0][0], [&](int r, int k) {
    return (r < hb && k < hb) ? F.get(i0 + r, i0 + k) : (r == k ? T(1) : T(0));
  });
  __syncthreads();
  for (int r = threadIdx.x; r < NB; r += 4 * NB) rcp[r] = pivot_rcp(D[r][r]);
  __syncthreads();
  masked_factor_copies<T, NB, 4 * NB>(D, rcp, LT, VT);
  __syncthreads();
  T *slot = dinv + (int64_t)blockIdx.x * 4 * NB * NB;
  triangle_inverses<T, NB, 4 * NB>(LT, VT, buf, rcp, slot);
  __syncthreads();  // the inverses are in global memory, visible to this CTA
  constexpr int TS = diag_tstride<T, NB>();
  const int nblk = ceil_div(n, NB);
#pragma unroll 1
  for (int side = 0; side < 2; ++side) {  // 0: L_bb^{-1} L_b,b-1   1: U_bb^{-1} U_b,b+1
    const int nb = (int)blockIdx.x + (side == 0 ? -1 : 1);
    T *out = slot + (2 + side) * NB * NB;
    if (nb < 0 || nb >= nblk) {
      for (int e = threadIdx.x; e < NB * NB; e += 4 * NB) out[e] = T(0);
      continue;
    }
    const int64_t j0 = (int64_t)nb * NB;
    const int hj = (int)min64(NB, n - j0);
    const T *inv = slot + side * NB * NB;
    stage_tile<NB, 4 * NB, TS>(LT, [&](int r, int k) { return inv[r * NB + k]; });
    stage_tile<NB, 4 * NB, TS>(VT, [&](int r, int k) { return (r < hb && k < hj) ? F.get(i0 + r, j0 + k) : T(0); });
    __syncthreads();
    tile_product<T, NB, TS>(LT, VT);
    for (int e = threadIdx.x; e < NB * NB; e += 4 * NB) out[e] = VT[(e / NB) * TS + e % NB];
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Published solution blocks: every entry of a finished block X_s goes out as
// 8-byte words {32 value bits, tag s + 1} (one word per binary32 value, two
// per binary64), written with single stores that are atomic as a whole.  A
// reader that sees the tag has the value: no fence on the writer's side and
// no separate flag to read first, so a block reaches the next step one L2
// round trip after it is stored.  The buffer is zeroed before each launch,
// so no tag survives from an earlier solve.
// ---------------------------------------------------------------------------
template <typename T>
struct XWords {
  static constexpr int W = sizeof(T) / 4;
};
__device__ __forceinline__ void xw_store(unsigned long long *p, uint32_t bits, uint32_t tag) {
  const unsigned long long v = ((unsigned long long)tag << 32) | bits;
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long xw_load(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void xw_put(unsigned long long *p, float v, uint32_t tag) {
  xw_store(p, __float_as_uint(v), tag);
}
__device__ __forceinline__ void xw_put(unsigned long long *p, double v, uint32_t tag) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  xw_store(p, (uint32_t)u, tag);
  xw_store(p + 1, (uint32_t)(u >> 32), tag);
}
// The value of an entry's words if every word carries tag.
__device__ __forceinline__ bool xw_decode(const unsigned long long (&w)[1], uint32_t tag, float &v) {
  v = __uint_as_float((uint32_t)w[0]);
  return (uint32_t)(w[0] >> 32) == tag;
}
__device__ __forceinline__ bool xw_decode(const unsigned long long (&w)[2], uint32_t tag, double &v) {
  v = __longlong_as_double((long long)(((w[1] & 0xFFFFFFFFull) << 32) | (w[0] & 0xFFFFFFFFull)));
  return (uint32_t)(w[0] >> 32) == tag && (uint32_t)(w[1] >> 32) == tag;
}
// One attempt: true (and the value) once every word of the entry carries tag.
__device__ __forceinline__ bool xw_try(const unsigned long long *p, uint32_t tag, float &v) {
  const unsigned long long w = xw_load(p);
  if ((uint32_t)(w >> 32) != tag) return false;
  v = __uint_as_float((uint32_t)w);
  return true;
}
__device__ __forceinline__ bool xw_try(const unsigned long long *p, uint32_t tag, double &v) {
  const unsigned long long w0 = xw_load(p), w1 = xw_load(p + 1);
  if ((uint32_t)(w0 >> 32) != tag || (uint32_t)(w1 >> 32) != tag) return false;
  v = __longlong_as_double((long long)(((w1 & 0xFFFFFFFFull) << 32) | (w0 & 0xFFFFFFFFull)));
  return true;
}
// Bounded wait for one entry, with the same limits and early exit as
// bounded_wait_geq.  On expiry records EBV_ERR_TIMEOUT with `where`.
template <typename T>
__device__ __forceinline__ bool xw_wait(const unsigned long long *p, uint32_t tag, T &v, DevStatus *st,
                                        int where) {
  for (long long it = 0; it < kSpinLimit; ++it) {
    if (xw_try(p, tag, v)) return true;
    if ((it & 255) == 255 && st && ld_acquire(&st->code) != 0) return false;
    if (it >= 32) __nanosleep(64);
  }
  set_status(st, EBV_ERR_TIMEOUT, where);
  return false;
}

// ---------------------------------------------------------------------------
// Block substitution in one cooperative launch per triangle (Eq. 1: LY = B,
// then UX = Y), left-looking.  Steps t = 0..nblk-1 visit the row blocks in
// solve order (increasing for L, decreasing for U); each chunk of RC
// right-hand sides is an independent chain of CTAs.  CTA h of a chain owns
// the steps t = h (mod G) and takes them in order: for its block t it folds
// the published blocks s < t-1 into a register accumulator, acc -= F(t,s)
// X_s, in the order they were published, applies the diagonal-block inverse
// (y = D_t^{-1} acc, a tile product) before block t-1 exists, and once X_{t-1}
// is there only does X_t = y - (D_t^{-1} F(t,t-1)) X_{t-1}, then publishes
// X_t (tagged words, above) and writes it to B.
// Rounding: the folds accumulate from zero and meet B_t once; the inverse's
// off-diagonal part and the coupling product accumulate from zero too, and
// the diagonal term D_t^{-1}(r, r) acc_r (of the size of the solution) joins
// last.  Every small term is then rounded against small partial sums, and an
// entry of X_t takes O(1) roundings at its own magnitude instead of one per
// folded product (for n = 16384 that is 16k roundings against a value of
// order 1, about 1e-14 of backward error).  Only the owner ever touches
// block t of B, and a CTA never works on a later block while its current one
// could advance, so the critical path per step is: X_{t-1}'s words seen ->
// one 64 x 64 x RC product -> X_t stored.
// The factor tiles F(t, s) and the coupling tile stream through an NS-stage
// shared-memory ring filled by 16-byte cp.async (16-byte chunks XOR-swizzled
// by row, so the fold's column reads hit distinct banks); band rows (not
// 16-byte aligned) by one-element cp.async, so the next tile's copy is in
// flight during the current fold instead of on the chain (the band's factors
// outgrow L2: one HBM round trip per serial load); views with computed
// entries by plain loads, all issued before the first store.  Published entries
// of an earlier block are taken with one attempt each; only if one is
// missing does thread 0 poll for the block (one poller per CTA at the front
// of the chain) before every thread waits for its own.  At the last step
// every thread waits for its entries of X_{t-1} directly.  Every wait is
// bounded and gives up once the workspace status reports an error.  All
// CTAs must be co-resident: the host code launches at most the occupancy limit,
// cooperatively.
// xw: nchunk * nblk * NB * RC entries of XWords<T>::W words, zeroed.
// Dynamic shared memory: trsvl_smem_bytes<T, NB, RC, NS>().
// ---------------------------------------------------------------------------
template <typename T, int NB>
__host__ __device__ constexpr int trsvl_stride() { return NB + 16 / (int)sizeof(T); }  // 16-byte rows

template <typename T, int NB, int RC, int NS>
constexpr size_t trsvl_smem_bytes() {
  return sizeof(T) * ((size_t)NS * NB * NB + (size_t)NB * trsvl_stride<T, NB>() + 3 * (size_t)NB * (RC + 1));
}

// Element (r, k) of a swizzled NB x NB ring tile.
template <typename T, int NB>
__device__ __forceinline__ int ring_idx(int r, int k) {
  constexpr int E = 16 / (int)sizeof(T), CPR = NB / E;  // elements per chunk, chunks per row
  return r * NB + (((k / E) ^ (r % CPR)) * E) + (k % E);
}

// Elements k .. k+3 (k a multiple of 4) of row r of a ring tile, as 16-byte loads.
template <int NB>
__device__ __forceinline__ void ring_ld4(const float *tile, int r, int k, float (&f)[4]) {
  const float4 v = *reinterpret_cast<const float4 *>(tile + ring_idx<float, NB>(r, k));
  f[0] = v.x, f[1] = v.y, f[2] = v.z, f[3] = v.w;
}
template <int NB>
__device__ __forceinline__ void ring_ld4(const double *tile, int r, int k, double (&f)[4]) {
  const double2 v0 = *reinterpret_cast<const double2 *>(tile + ring_idx<double, NB>(r, k));
  const double2 v1 = *reinterpret_cast<const double2 *>(tile + ring_idx<double, NB>(r, k + 2));
  f[0] = v0.x, f[1] = v0.y, f[2] = v1.x, f[3] = v1.y;
}
// acc[q] -= sum_k P(r_q, k) xs[k][tc] over a ring tile P, r_q = tr + PASS q.
template <typename T, int NB, int RC, int PASS, int OPT>
__device__ __forceinline__ void ring_fold(const T *P, const T (*xs)[RC + 1], int tr, int tc, T (&acc)[OPT]) {
#pragma unroll 4
  for (int k = 0; k < NB; k += 4) {
    T x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) x[u] = xs[k + u][tc];
#pragma unroll
    for (int q = 0; q < OPT; ++q) {
      T f[4];
      ring_ld4<NB>(P, tr + PASS * q, k, f);
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[q] -= f[u] * x[u];
    }
  }
}

template <typename T, int NB, int RC, bool UPPER, int NS, int MINB, bool XV = false>
__global__ void __launch_bounds__(256, MINB) k_trsv_left(MatView<T, XV> F, int64_t n, T *B, int64_t ldb, int nrhs,
                                                         const T *dinv, unsigned long long *xw, DevStatus *st) {
  constexpr int NT = 256, DS = trsvl_stride<T, NB>(), E = 16 / (int)sizeof(T), CPR = NB / E;
  constexpr int PASS = NT / RC, OPT = NB / PASS;
  static_assert(NT % RC == 0 && NB % PASS == 0 && NS >= 2, "shape");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *Fr = reinterpret_cast<T *>(smem_raw);                                           // NS ring tiles
  T(*Di)[DS] = reinterpret_cast<T(*)[DS]>(Fr + NS * NB * NB);                          // D_t^{-1}
  T(*Xs)[NB][RC + 1] = reinterpret_cast<T(*)[NB][RC + 1]>(Fr + NS * NB * NB + NB * DS);  // 2 x X_s
  T(*Ac)[RC + 1] = reinterpret_cast<T(*)[RC + 1]>(Fr + NS * NB * NB + NB * DS + 2 * NB * (RC + 1));
  __shared__ T dg[NB];  // diagonal of D_t^{-1} (Di holds the rest, zero diagonal)
  if (st && st->done) return;  // refinement already converged
  const int nblk = ceil_div(n, NB);
  const int nchunk = ceil_div(nrhs, RC);
  const int chunk = blockIdx.x % nchunk, h = blockIdx.x / nchunk;
  const int G = gridDim.x / nchunk;
  if (h >= G) return;
  const int c0 = chunk * RC, wc = min(RC, nrhs - c0);
  unsigned long long *xc = xw + (size_t)chunk * nblk * NB * RC * XWords<T>::W;
  auto xent = [&](int s, int k, int c) { return xc + (((size_t)s * NB + k) * RC + c) * XWords<T>::W; };
  auto blk = [&](int s) { return UPPER ? nblk - 1 - s : s; };
  auto rows_of = [&](int s) { return (int)min64(NB, n - (int64_t)blk(s) * NB); };
  // Blocks s >= t - reach couple into block t (a band limits reach).
  const int reach = (int)max64(1, min64((UPPER ? F.ku + NB - 1 : F.kl + NB - 1) / NB, (int64_t)nblk));
  const int tc = threadIdx.x % RC, tr = threadIdx.x / RC;
  // plain dense storage: tiles copied as they are (a lower-triangle view reads U through get())
  const bool direct = !XV && F.kl >= kDenseBand && F.ku >= kDenseBand && F.ld % E == 0 &&
                      ((uintptr_t)F.base % 16) == 0;

  // Ring tile j of block t: F(t, sb + j) for j < m, then the coupling tile.
  auto load_tile = [&](T *dst, int t, int s, const T *g) {
    if (g) {
      for (int e = threadIdx.x; e < NB * CPR; e += NT) {
        const int r = e / CPR, c = e % CPR;
        cp_async16(dst + ring_idx<T, NB>(r, c * E), g + r * NB + c * E, 16);
      }
      return;
    }
    const int64_t i0 = (int64_t)blk(t) * NB, j0 = (int64_t)blk(s) * NB;
    const int hi = rows_of(t), hj = rows_of(s);
    if (direct) {
      for (int e = threadIdx.x; e < NB * CPR; e += NT) {
        const int r = e / CPR, c = e % CPR;
        const int valid = r < hi ? max(0, min(E, hj - c * E)) : 0;
        cp_async16(dst + ring_idx<T, NB>(r, c * E), valid ? F.base + (i0 + r) * F.ld + j0 + c * E : F.base,
                   valid * (int)sizeof(T));
      }
    } else if constexpr (!XV) {
      // band rows (and dense rows of an odd ld): entry (i, j) at base + i ld + j
      // inside the band, contiguous along a row but not 16-byte aligned; one
      // element per copy, zero-filled outside the band and the matrix
      for (int e = threadIdx.x; e < NB * NB; e += NT) {
        const int r = e / NB, k = e % NB;
        const int64_t i = i0 + r, j = j0 + k;
        const bool ok = r < hi && k < hj && F.in(i, j);
        cp_async_el(dst + ring_idx<T, NB>(r, k), ok ? F.base + i * F.ld + j : F.base, ok ? (int)sizeof(T) : 0);
      }
    } else {
      // views with computed entries: every load of the tile in flight before the first store
      T v[NB * NB / NT];
#pragma unroll
      for (int q = 0; q < NB * NB / NT; ++q) {
        const int e = threadIdx.x + NT * q, r = e / NB, k = e % NB;
        v[q] = (r < hi && k < hj) ? F.get(i0 + r, j0 + k) : T(0);
      }
#pragma unroll
      for (int q = 0; q < NB * NB / NT; ++q) {
        const int e = threadIdx.x + NT * q;
        dst[ring_idx<T, NB>(e / NB, e % NB)] = v[q];
      }
    }
  };
  auto commit = [] { asm volatile("cp.async.commit_group;" ::: "memory"); };
  // every copy of this thread landed (also before giving up: none stays in flight)
  auto drain = [] { asm volatile("cp.async.wait_group 0;" ::: "memory"); };
  // X_s into xs: one attempt at every entry of this thread (zero outside the
  // block / chunk).  All loads are issued before any tag is checked, so an
  // attempt costs one memory round trip however many entries a thread has.
  auto try_x = [&](int s, T (*xs)[RC + 1]) -> bool {
    const uint32_t tag = (uint32_t)s + 1;
    const int hj = rows_of(s);
    unsigned long long wv[OPT][XWords<T>::W];
#pragma unroll
    for (int j = 0; j < OPT; ++j) {
      const int k = tr + PASS * j;
#pragma unroll
      for (int u = 0; u < XWords<T>::W; ++u)
        wv[j][u] = (k < hj && tc < wc) ? xw_load(xent(s, k, tc) + u) : ((unsigned long long)tag << 32);
    }
    bool ok = true;
#pragma unroll
    for (int j = 0; j < OPT; ++j) {
      const int k = tr + PASS * j;
      T v;
      if (!xw_decode(wv[j], tag, v)) ok = false;
      xs[k][tc] = (k < hj && tc < wc) ? v : T(0);
    }
    return ok;
  };
  // Bounded wait for all of this thread's entries of X_s (limits and early
  // exit as bounded_wait_geq; on expiry records EBV_ERR_TIMEOUT with s).
  auto wait_x = [&](int s, T (*xs)[RC + 1]) -> bool {
    for (long long it = 0; it < kSpinLimit; ++it) {
      if (try_x(s, xs)) return true;
      if ((it & 255) == 255 && st && ld_acquire(&st->code) != 0) return false;
      if (it >= 32) __nanosleep(64);
    }
    set_status(st, EBV_ERR_TIMEOUT, s);
    return false;
  };

  for (int t = h; t < nblk; t += G) {
    const int64_t i0 = (int64_t)blk(t) * NB;
    const int hi = rows_of(t);
    const int sb = max(0, t - reach);
    const int m = max(0, t - 1 - sb);           // folded blocks s = sb .. t-2
    const int ntiles = m + (t >= 1 ? 1 : 0);    // + the coupling tile
    const T *slot = dinv + (int64_t)blk(t) * 4 * NB * NB;
    const T *gmat = slot + (UPPER ? 3 : 2) * NB * NB;  // D_t^{-1} F(t, t-1)
    auto tile = [&](int j) {
      if (j < ntiles) load_tile(Fr + (j % NS) * NB * NB, t, sb + j, j < m ? nullptr : gmat);
      commit();
    };
    // (the ring, Di, Xs and Ac are free: the previous block ended with a
    // barrier after its last use of them)
    for (int j = 0; j < NS - 1; ++j) tile(j);
    stage_tile<NB, NT, DS>(&Di[0][0], [&](int r, int k) {
      return r == k ? T(0) : slot[(UPPER ? NB * NB : 0) + r * NB + k];
    });
    for (int r = threadIdx.x; r < NB; r += NT) dg[r] = slot[(UPPER ? NB * NB : 0) + r * NB + r];
    T acc[OPT];
#pragma unroll
    for (int q = 0; q < OPT; ++q) {
      const int r = tr + PASS * q;
      Ac[r][tc] = (r < hi && tc < wc) ? B[(i0 + r) * ldb + c0 + tc] : T(0);  // B_t, joined after the folds
      acc[q] = T(0);
    }
    for (int j = 0; j < m; ++j) {
      const int s = sb + j;
      T(*xs)[RC + 1] = Xs[j & 1];
      const bool got = try_x(s, xs);
      asm volatile("cp.async.wait_group %0;" ::"n"(NS - 2) : "memory");
      if (__syncthreads_or(!got)) {  // X_s not (fully) there yet
        bool ok = true;
        if (threadIdx.x == 0) {
          T v;
          ok = xw_wait(xent(s, 0, 0), (uint32_t)s + 1, v, st, s);
        }
        if (__syncthreads_or(!ok)) return drain();
        ok = wait_x(s, xs);
        if (__syncthreads_or(!ok)) return drain();
      }
      tile(j + NS - 1);  // into the stage every thread finished with before the barrier
      ring_fold<T, NB, RC, PASS, OPT>(Fr + (j % NS) * NB * NB, xs, tr, tc, acc);
    }
    // y = D_t^{-1} (B_t + acc), before block t-1 is needed: the off-diagonal
    // part now, the diagonal term after the coupling product.
#pragma unroll
    for (int q = 0; q < OPT; ++q) Ac[tr + PASS * q][tc] += acc[q];  // this thread's own entries
    __syncthreads();
    // D_t^{-1} is triangular (Di: lower for L, upper for U, zero diagonal):
    // a group of four columns k .. k+3 is skipped for pass q when it holds
    // no entry of any of the warp's rows (warp-uniform; an FP64 warp
    // instruction costs its pipe slot whatever its lanes do).
    const int wr0 = (threadIdx.x & ~31) / RC, wr1 = (threadIdx.x | 31) / RC;  // the warp's tr range
    T y[OPT];
#pragma unroll
    for (int q = 0; q < OPT; ++q) y[q] = T(0);
#pragma unroll 4
    for (int k = 0; k < NB; k += 4) {
      T x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) x[u] = Ac[k + u][tc];
#pragma unroll
      for (int q = 0; q < OPT; ++q) {
        if (UPPER ? k + 3 <= wr0 + PASS * q : k >= wr1 + PASS * q) continue;
        const T *d = &Di[tr + PASS * q][k];
        T f[4];
        if constexpr (sizeof(T) == 4) {
          const float4 v = *reinterpret_cast<const float4 *>(d);
          f[0] = v.x, f[1] = v.y, f[2] = v.z, f[3] = v.w;
        } else {
          const double2 v0 = *reinterpret_cast<const double2 *>(d), v1 = *reinterpret_cast<const double2 *>(d + 2);
          f[0] = v0.x, f[1] = v0.y, f[2] = v1.x, f[3] = v1.y;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) y[q] += f[u] * x[u];
      }
    }
    if (t >= 1) {  // x_t = y - (D_t^{-1} F(t, t-1)) x_{t-1}
      T(*xs)[RC + 1] = Xs[m & 1];
      const bool ok = wait_x(t - 1, xs);
      drain();
      if (__syncthreads_or(!ok)) return;
      ring_fold<T, NB, RC, PASS, OPT>(Fr + (m % NS) * NB * NB, xs, tr, tc, y);
    }
#pragma unroll
    for (int q = 0; q < OPT; ++q) {
      const int r = tr + PASS * q;
      y[q] += dg[r] * Ac[r][tc];
    }
    const uint32_t tag = (uint32_t)t + 1;
#pragma unroll
    for (int q = 0; q < OPT; ++q) {
      const int r = tr + PASS * q;
      if (r < hi && tc < wc) {
        xw_put(xent(t, r, tc), y[q], tag);
        B[(i0 + r) * ldb + c0 + tc] = y[q];
      }
    }
    __syncthreads();  // the ring, Di, Xs and Ac are free for the next block
  }
  drain();
}

// ---------------------------------------------------------------------------
// Small systems (n <= kSmallSolveMaxN): LY = B then UX = Y (Eq. 1) by one CTA
// of 8 warps, 32-row blocks.  Per block: 8 threads share each row's sum over
// the finished blocks (strided columns, four independent partial sums so all
// loads of a block are in flight at once, shuffle reduction; accumulated
// from zero and subtracted from b once), then warp 0 solves the
// 32 x 32 diagonal block, lane l holding row r0+l's block entries in
// registers and the solved values passed by shuffle.  No inverse of any
// diagonal block is formed.  Right-hand sides one column at a time.
// ---------------------------------------------------------------------------
constexpr int kSmallSolveMaxN = 512;

template <typename T>
__global__ void __launch_bounds__(256) k_small_solve(MatView<T> F, int n, T *B, int64_t ldb, int nrhs) {
  __shared__ T ys[kSmallSolveMaxN];
  __shared__ T acc[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rq = threadIdx.x >> 3, part = threadIdx.x & 7;  // 8 threads per row of a block
  const int nb = (n + 31) / 32;
  for (int c = 0; c < nrhs; ++c) {
    for (int i = threadIdx.x; i < n; i += 256) ys[i] = B[(int64_t)i * ldb + c];
    __syncthreads();
    // forward: unit lower L, y overwrites ys
    for (int blk = 0; blk < nb; ++blk) {
      const int r0 = 32 * blk;
      {
        const int r = r0 + rq, j1 = r0;
        T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
        if (r < n)
          for (int j = part; j < j1; j += 32) {
            s0 += F.get(r, j) * ys[j];
            if (j + 8 < j1) s1 += F.get(r, j + 8) * ys[j + 8];
            if (j + 16 < j1) s2 += F.get(r, j + 16) * ys[j + 16];
            if (j + 24 < j1) s3 += F.get(r, j + 24) * ys[j + 24];
          }
        T sum = (s0 + s1) + (s2 + s3);
        for (int off = 4; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
        if (part == 0) acc[rq] = (r < n) ? ys[r] - sum : T(0);
      }
      __syncthreads();
      if (warp == 0) {
        const int rl = r0 + lane;
        T lrow[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) lrow[k] = (rl < n && k < lane && r0 + k < n) ? F.get(rl, r0 + k) : T(0);
        T v = acc[lane];
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          const T yk = __shfl_sync(0xffffffffu, v, k);
          if (lane > k) v -= lrow[k] * yk;
        }
        if (rl < n) ys[rl] = v;
      }
      __syncthreads();
    }
    // backward: U with its diagonal, x overwrites ys
    for (int blk = nb - 1; blk >= 0; --blk) {
      const int r0 = 32 * blk, rend = min(n, r0 + 32);
      {
        const int r = r0 + rq;
        T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
        if (r < n)
          for (int j = rend + part; j < n; j += 32) {
            s0 += F.get(r, j) * ys[j];
            if (j + 8 < n) s1 += F.get(r, j + 8) * ys[j + 8];
            if (j + 16 < n) s2 += F.get(r, j + 16) * ys[j + 16];
            if (j + 24 < n) s3 += F.get(r, j + 24) * ys[j + 24];
          }
        T sum = (s0 + s1) + (s2 + s3);
        for (int off = 4; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
        if (part == 0) acc[rq] = (r < n) ? ys[r] - sum : T(0);
      }
      __syncthreads();
      if (warp == 0) {
        const int rl = r0 + lane;
        T urow[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) urow[k] = (rl < n && k > lane && r0 + k < n) ? F.get(rl, r0 + k) : T(0);
        const T rc = rl < n ? pivot_rcp(F.get(rl, rl)) : T(0);
        T v = acc[lane];
#pragma unroll
        for (int k = 31; k >= 0; --k) {
          if (lane == k) v *= rc;
          const T xk = __shfl_sync(0xffffffffu, v, k);
          if (lane < k) v -= urow[k] * xk;
        }
        if (rl < n) ys[rl] = v;
      }
      __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += 256) B[(int64_t)i * ldb + c] = ys[i];
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Iterative refinement helpers.
// ---------------------------------------------------------------------------

// Split a binary64 value into two binary32 values with a = hi + lo up to
// 2^-47 |a|, using integer operations only (the FP64 pipe is the scarce unit
// on this GPU).  hi is a with its significand truncated to 24 bits; lo is the
// remainder rounded to binary32.  Magnitudes below 2^-126 map to 0 (their
// contribution to a residual of an O(1) system is below 1e-37).
__device__ __forceinline__ void split_f64(double a, float &hi, float &lo) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(a);
  const unsigned int sign = (unsigned int)(u >> 32) & 0x80000000u;
  const int ebias = (int)((u >> 52) & 0x7FF);
  const int e = ebias - 1023;
  if (ebias == 0x7FF) {  // inf / nan
    hi = __int_as_float(sign | 0x7F800000u | (((u << 12) != 0) ? 0x400000u : 0u));
    lo = 0.f;
    return;
  }
  if (e < -126) {
    hi = 0.f;
    lo = 0.f;
    return;
  }
  if (e > 127) {
    hi = __int_as_float(sign | 0x7F800000u);
    lo = 0.f;
    return;
  }
  const unsigned long long m = u & 0xFFFFFFFFFFFFFull;
  hi = __int_as_float(sign | ((unsigned int)(e + 127) << 23) | (unsigned int)(m >> 29));
  const unsigned int rem = (unsigned int)(m & 0x1FFFFFFFull);
  float l = __uint2float_rn(rem) * 2.220446049250313e-16f;  // * 2^-52, exact
  l = l * __int_as_float((unsigned int)(e + 127) << 23);    // * 2^e
  lo = sign ? -l : l;
}

// hi/lo planes of X (n x nrhs, FP64, ldx) for the residual kernel.
__global__ void k_split_x(const double *x, int64_t ldx, int64_t n, int nrhs, float *xhi, float *xlo,
                          const DevStatus *st) {
  if (st && st->done) return;
  const int64_t total = n * nrhs;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / nrhs;
    const int c = (int)(e % nrhs);
    const double v = x[i * ldx + c];
    const float h = __double2float_rn(v);
    xhi[e] = h;
    xlo[e] = __double2float_rn(v - (double)h);
  }
}

// R = B - A X with A in FP64, evaluated in binary32 multi-word arithmetic
// (TripleF above) so the FP64 ALU, ~75x slower than
// FP32 on GB300, is touched once per output.  CTA tile: RB rows x RC
// right-hand sides; K staged through shared memory in KC-wide slabs, the next
// slab's loads in flight while the current one is consumed.  Also folds
// max_i |R_ic| per column into rmax (as ordered bit patterns).
template <int RB, int RC, int KC>
__global__ void __launch_bounds__(256, 4)
    k_residual_df(const double *A, int64_t lda, int64_t n, const float *xhi, const float *xlo, int nrhs,
                  const double *B, int64_t ldb, double *R, int64_t ldr, unsigned long long *rmax,
                  const DevStatus *st) {
  constexpr int NT = 256;
  constexpr int ROWS_PER_PASS = NT / RC;
  constexpr int OPT = RB / ROWS_PER_PASS;  // outputs per thread
  constexpr int LA = RB * KC / NT, LX = KC * RC / NT;
  static_assert(NT % RC == 0 && RB % ROWS_PER_PASS == 0, "shape");
  static_assert(LA * NT == RB * KC && LX * NT == KC * RC, "slab must divide evenly");
  __shared__ float ah[RB][KC + 1], al[RB][KC + 1];
  __shared__ float xh[KC][RC + 1], xl[KC][RC + 1];
  __shared__ unsigned long long cmax[RC];
  if (st && st->done) return;
  const int64_t r0 = (int64_t)blockIdx.x * RB;
  const int c0 = blockIdx.y * RC;
  const int c = threadIdx.x % RC;
  const int rr = threadIdx.x / RC;
  TripleF acc[OPT];
#pragma unroll
  for (int q = 0; q < OPT; ++q) acc[q].zero();
  if (threadIdx.x < RC) cmax[threadIdx.x] = 0ull;
  double pa[LA];
  float pxh[LX], pxl[LX];
  auto fetch = [&](int64_t k0) {
#pragma unroll
    for (int u = 0; u < LA; ++u) {
      const int e = threadIdx.x + NT * u, i = e / KC, k = e % KC;
      const int64_t gi = r0 + i, gk = k0 + k;
      pa[u] = (gi < n && gk < n) ? A[gi * lda + gk] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < LX; ++u) {
      const int e = threadIdx.x + NT * u, k = e / RC, cc = e % RC;
      const int64_t gk = k0 + k;
      const bool ok = gk < n && c0 + cc < nrhs;
      pxh[u] = ok ? xhi[gk * nrhs + c0 + cc] : 0.f;
      pxl[u] = ok ? xlo[gk * nrhs + c0 + cc] : 0.f;
    }
  };
  fetch(0);
  for (int64_t k0 = 0; k0 < n; k0 += KC) {
    __syncthreads();  // the previous slab has been consumed
#pragma unroll
    for (int u = 0; u < LA; ++u) {
      const int e = threadIdx.x + NT * u;
      split_f64(pa[u], ah[e / KC][e % KC], al[e / KC][e % KC]);
    }
#pragma unroll
    for (int u = 0; u < LX; ++u) {
      const int e = threadIdx.x + NT * u;
      xh[e / RC][e % RC] = pxh[u];
      xl[e / RC][e % RC] = pxl[u];
    }
    __syncthreads();
    if (k0 + KC < n) fetch(k0 + KC);
#pragma unroll 4
    for (int k = 0; k < KC; ++k) {
      const float xhk = xh[k][c], xlk = xl[k][c];
#pragma unroll
      for (int q = 0; q < OPT; ++q) {
        const int i = rr + q * ROWS_PER_PASS;
        acc[q].fma_split(ah[i][k], al[i][k], xhk, xlk);
      }
    }
  }
  double dmax = 0.0;
#pragma unroll
  for (int q = 0; q < OPT; ++q) {
    const int64_t gi = r0 + rr + q * ROWS_PER_PASS;
    if (gi < n && c0 + c < nrhs) {
      const double rv = B[gi * ldb + c0 + c] - acc[q].value();
      R[gi * ldr + c0 + c] = rv;
      dmax = fmax(dmax, fabs(rv));
    }
  }
  atomicMax(&cmax[c], (unsigned long long)__double_as_longlong(dmax));
  __syncthreads();
  if (threadIdx.x < RC && c0 + threadIdx.x < nrhs) atomicMax(&rmax[c0 + threadIdx.x], cmax[threadIdx.x]);
}

// max_i |B_ic| per column (ordered bit patterns).
__global__ void k_colmax(const double *B, int64_t ldb, int64_t n, int nrhs, unsigned long long *out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * nrhs; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / nrhs;
    const int c = (int)(e % nrhs);
    atomicMax(&out[c], (unsigned long long)__double_as_longlong(fabs(B[i * ldb + c])));
  }
}

// Stop test of refinement step `it` (0 = residual of the unrefined solution).
__global__ void k_ir_check(const unsigned long long *rmax, const unsigned long long *bmax, int nrhs, int it,
                           int max_iter, double tol, DevStatus *st, ebv_refine_report_t *rep) {
  if (st->done) return;
  double rel = 0.0;
  for (int c = 0; c < nrhs; ++c) {
    const double r = __longlong_as_double((long long)rmax[c]);
    const double bb = __longlong_as_double((long long)bmax[c]);
    const double q = bb > 0.0 ? r / bb : r;
    rel = (q > rel || q != q) ? q : rel;
  }
  if (rep) {
    if (it == 0) rep->resid_first = rel;
    rep->resid_final = rel;
    rep->iters = it;
  }
  const bool conv = rel <= tol;
  if (conv || it >= max_iter) {
    st->done = 1;
    if (rep) rep->status = conv ? EBV_OK : EBV_ERR_NOT_CONVERGED;
  }
}

// dst(n x nrhs, T) = (T) src (FP64), skipped once refinement has converged.
template <typename T>
__global__ void k_narrow(const double *src, int64_t lds, T *dst, int64_t ldd, int64_t n, int nrhs,
                         const DevStatus *st) {
  if (st && st->done) return;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * nrhs; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / nrhs;
    const int c = (int)(e % nrhs);
    dst[i * ldd + c] = (T)src[i * lds + c];
  }
}

// x (FP64) = d, or x += d when accumulate; skipped once converged.
template <typename T>
__global__ void k_update_x(double *x, int64_t ldx, const T *d, int64_t ldd, int64_t n, int nrhs, int accumulate,
                           const DevStatus *st) {
  if (st && st->done) return;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * nrhs; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / nrhs;
    const int c = (int)(e % nrhs);
    const double v = (double)d[i * ldd + c];
    x[i * ldx + c] = accumulate ? x[i * ldx + c] + v : v;
  }
}

}  // namespace
}  // namespace ebv
