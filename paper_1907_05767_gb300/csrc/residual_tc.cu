// FP64-accurate residual R = B - A X of the refinement loop on the tensor
// cores, by exact splitting into small integers (the Ozaki scheme).
//
// Row i of A is written in fixed point against its own power of two,
// |a_ij| < 2^E_i:  a_ij ~ Q_ij 2^(E_i - 59) with the integer
// Q_ij = trunc(a_ij 2^(59 - E_i)), |Q_ij| < 2^59, and Q_ij is cut into ten
// balanced base-64 digits, Q_ij = sum_s d_s 2^(54 - 6s), d_s in [-33, 32].
// Column c of X likewise against 2^F_c with digits e_t.  Every digit is an
// integer of at most 6 bits plus sign, exact in bfloat16, so each digit
// pair (s, t) contributes an exact integer product to
//
//   (A X)_ic = 2^(E_i + F_c - 10) sum_{s,t} 2^(-6(s+t)) sum_j d_s(a_ij) e_t(x_jc).
//
// The pairs with s + t = d (d = 0..9, 55 pairs) share one FP32 accumulator
// in TMEM; with |d_s e_t| <= 33^2 and at most 10 pairs per diagonal, 1024
// columns of j keep every partial sum an integer below 2^24, so the tensor
// cores add exactly.  Every 1024 columns the ten diagonal sums are drained
// into a triple-binary32 accumulator per output (scaled by 2^(-6d), exact).
// Dropped: pairs with s + t >= 10 (weight <= 2^-60 of the leading pair) and
// the truncation of A and X below 2^-59 of their row / column scale, so the
// result is accurate to ~2^-50 of (max_j |a_ij|) (max_j |x_jc|) n^(1/2) for
// random-signed data -- well below the 2^-44 sum_j |a_ij x_jc| the refinement
// needs for the systems it targets (rows whose largest entry is comparable
// to their dot product, as in diagonally dominant A).
//
// Kernel (one CTA per 128 rows x 32 right-hand sides, 21 warps):
//   warps 5..20  convert: FP64 tile of A (128 x 32 per stage) -> ten digit
//                planes in shared memory, 64-byte swizzled K-major rows
//                (their first thread also TMA-loads the stage's X planes);
//   warp 4       allocates TMEM and issues, per stage and A digit, one MMA
//                over all its X digits (M=128, N<=256, K=16: 24 per stage);
//   warps 0..3   drain the ten diagonals every 1024 columns (TMEM lane =
//                row) and write R = B - A X and the column maxima of |R|.
// Two stages of 100 KB; every mbarrier wait is bounded.
#include <cuda.h>

#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "multiword.cuh"
#include "tcgen05.cuh"

namespace ebv {

namespace {

constexpr int RT_M = 128;       // rows per CTA (TMEM lanes)
constexpr int RT_N = 32;        // right-hand sides per CTA
constexpr int RT_K = 32;        // columns of A per stage (one 64-byte swizzle row)
constexpr int RT_S = 10;        // digit planes of A and of X
constexpr int RT_D = 10;        // diagonals s + t = 0 .. RT_D-1
constexpr int RT_CHUNK = 1024;  // columns per exact TMEM accumulation
constexpr int RT_STAGES = 2;
constexpr int RT_EPI_WARPS = 4, RT_MMA_WARP = 4, RT_CONV_WARP0 = 5, RT_CONV_WARPS = 16;
constexpr int RT_THREADS = 32 * (RT_CONV_WARP0 + RT_CONV_WARPS);
constexpr int RT_CONV_THREADS = 32 * RT_CONV_WARPS;
constexpr int RT_JOBS = RT_M * (RT_K / 8) / RT_CONV_THREADS;  // 8-column row pieces per converter thread
static_assert(RT_JOBS * RT_CONV_THREADS == RT_M * (RT_K / 8), "converter jobs must divide evenly");
constexpr int RT_APLANE = RT_M * RT_K * 2;  // 8 KB
constexpr int RT_XPLANE = RT_N * RT_K * 2;  // 2 KB
constexpr int RT_STAGE_BYTES = RT_S * (RT_APLANE + RT_XPLANE);
constexpr int RT_BAR_BYTES = 512;                   // mbarriers, TMEM address, flags, column maxima
constexpr int RT_SMEM = 1024 /* alignment slack */ + RT_STAGES * RT_STAGE_BYTES + RT_BAR_BYTES;
constexpr int RT_TM_H = RT_D * RT_N, RT_TM_M = RT_TM_H + RT_N, RT_TM_L = RT_TM_M + RT_N;  // accumulator words
constexpr int RT_TMEM_COLS = 512;
constexpr int kNonFinite = 1 << 20;  // exponent flag of a row / column holding Inf or NaN
static_assert((RT_D + 3) * RT_N <= RT_TMEM_COLS, "diagonal and output accumulators must fit in TMEM");
static_assert(RT_CHUNK % RT_K == 0, "chunk = whole stages");

// 32 * (2^48 + 2^42 + ... + 2^0): adding it turns the low nine base-64 digits
// of a two's complement value into u_s = d_s + 32 in [0, 63].
constexpr long long kDigitBias = 32LL * ((1LL << 48) + (1LL << 42) + (1LL << 36) + (1LL << 30) + (1LL << 24) +
                                         (1LL << 18) + (1LL << 12) + (1LL << 6) + 1LL);

// Biased binary exponent field of a double (0 for zero / subnormal, 2047 for
// Inf / NaN); |a| < 2^(field - 1022) for every finite a.
__device__ __forceinline__ int exp_field(double a) {
  return (int)((unsigned long long)__double_as_longlong(a) >> 52) & 0x7FF;
}

// Q = trunc(a 2^(59 - E)) for |a| < 2^E, E = field_max - 1022, i.e. the
// mantissa shifted by (field - field_max + 6) <= 6 places.
__device__ __forceinline__ long long fixed59(double a, int fmax) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(a);
  const int be = (int)(b >> 52) & 0x7FF;
  unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  int e = be;
  if (be) m |= 1ull << 52;
  else e = 1;
  const int sh = min(e - fmax + 6, 6);
  const unsigned long long mag = sh >= 0 ? (m << sh) : (sh > -64 ? (m >> -sh) : 0ull);
  return (b >> 63) ? -(long long)mag : (long long)mag;
}

// Balanced digit s of Q (digit 0 most significant) from qb = Q + kDigitBias,
// as a float (exact).  u = d + 32 in [0, 64] becomes a float without a
// conversion instruction: the bits 0x4B000000 | u are the float 2^23 + u.
__device__ __forceinline__ float digit_of(long long qb, int s) {
  const unsigned int u = s == 0 ? (unsigned int)((int)(qb >> 54) + 32)
                                : (unsigned int)((unsigned long long)qb >> (54 - 6 * s)) & 63u;
  return __uint_as_float(0x4B000000u | u) - 8388640.f;  // - (2^23 + 32)
}
// All ten digits of Q.
__device__ __forceinline__ void digits10(long long q, float (&d)[RT_S]) {
  const long long qb = q + kDigitBias;
#pragma unroll
  for (int s = 0; s < RT_S; ++s) d[s] = digit_of(qb, s);
}

// v * 2^k, exact while the result is a normal double; three factors keep
// each power of two inside the normal range for |k| <= 3066.
__device__ __forceinline__ double pow2(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }
__device__ __forceinline__ double times_pow2(double v, int k) {
  const int k1 = k / 3, k2 = (k - k1) / 2, k3 = k - k1 - k2;
  return v * pow2(k1) * pow2(k2) * pow2(k3);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&v);
}

// Byte offset of the 16-byte chunk `c16` (0..3) of row r in a 64-byte
// swizzled K-major tile (Swizzle<2,4,3>: address bits [4,5] ^= bits [7,8]).
__device__ __forceinline__ uint32_t sw64_offset(int r, int c16) { return r * 64 + ((c16 ^ ((r >> 1) & 3)) << 4); }

// ---------------------------------------------------------------------------
// Per-row maximum exponent field of A (once per solve; A does not change
// between refinement steps).
// ---------------------------------------------------------------------------
__global__ void k_row_expmax(const double *A, int64_t lda, int64_t n, int *rexp) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (i >= n) return;
  int m = 0;
  for (int64_t j = lane; j < n; j += 32) m = max(m, exp_field(A[i * lda + j]));
  for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
  if (lane == 0) rexp[i] = m == 2047 ? kNonFinite : m;
}

// Per-column maximum exponent field of X (cexp zeroed beforehand): one row
// per thread, a warp maximum per column, one atomic per warp and column.
__global__ void k_col_expmax(const double *X, int64_t ldx, int64_t n, int nrhs, int *cexp) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int c = 0; c < nrhs; ++c) {
    int f = k < n ? exp_field(X[k * ldx + c]) : 0;
    f = f == 2047 ? kNonFinite : f;
    for (int off = 16; off > 0; off >>= 1) f = max(f, __shfl_xor_sync(0xffffffffu, f, off));
    if ((threadIdx.x & 31) == 0 && f > 0) atomicMax(&cexp[c], f);
  }
}

// Digit planes of X: xp[((rb * RT_S + t) * RT_N + c) * npad + k] = e_t(x_k,
// rb*32 + c), zero for k >= n and for columns >= nrhs.
__global__ void k_x_planes(const double *X, int64_t ldx, int64_t n, int64_t npad, int nrhs, int nrb,
                           const int *cexp, __nv_bfloat16 *xp) {
  const int64_t total = npad * (int64_t)nrb * RT_N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = e % npad;
    const int cc = (int)(e / npad);  // rb * 32 + c
    const int rb = cc / RT_N, c = cc % RT_N;
    float d[RT_S];
    const bool ok = k < n && cc < nrhs && cexp[cc] < kNonFinite;
    if (ok) {
      digits10(fixed59(X[k * ldx + cc], cexp[cc]), d);
    } else {
#pragma unroll
      for (int t = 0; t < RT_S; ++t) d[t] = 0.f;
    }
#pragma unroll
    for (int t = 0; t < RT_S; ++t) xp[(((int64_t)rb * RT_S + t) * RT_N + c) * npad + k] = __float2bfloat16_rn(d[t]);
  }
}


// ---------------------------------------------------------------------------
// The residual kernel.  grid = (ceil(n / 128), ceil(nrhs / 32)).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(RT_THREADS, 1)
    k_residual_tc(const __grid_constant__ CUtensorMap tmX, const double *A, int64_t lda, int64_t n, int nrhs,
                  const int *rexp, const int *cexp, const double *B, int64_t ldb, double *R, int64_t ldr,
                  unsigned long long *rmax, int vec, DevStatus *st) {
  extern __shared__ uint8_t smem_raw[];
  if (st && st->done) return;  // refinement converged: nothing to evaluate
  uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *full = (uint64_t *)(base + RT_STAGES * RT_STAGE_BYTES);
  uint64_t *empty = full + RT_STAGES;
  uint64_t *tfull = empty + RT_STAGES;
  uint64_t *tempty = tfull + 1;
  uint32_t *tmem_holder = (uint32_t *)(tempty + 1);
  volatile int *abort_flag = (volatile int *)(tmem_holder + 1);
  unsigned long long *cmax = (unsigned long long *)(base + RT_STAGES * RT_STAGE_BYTES + 64);  // RT_N entries
  auto a_plane = [&](int s, int p) { return base + s * RT_STAGE_BYTES + p * RT_APLANE; };
  auto x_plane = [&](int s, int p) { return base + s * RT_STAGE_BYTES + RT_S * RT_APLANE + p * RT_XPLANE; };

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t r0 = (int64_t)blockIdx.x * RT_M;
  const int cb = blockIdx.y;
  const int nst = ceil_div(n, RT_K);  // stages
  constexpr int SPC = RT_CHUNK / RT_K;  // stages per chunk
  const int nchunk = ceil_div(nst, SPC);

  if (threadIdx.x == 0) {
    for (int s = 0; s < RT_STAGES; ++s) {
      mbar_init(&full[s], RT_CONV_THREADS + 1);  // converters + the X planes' expect_tx
      mbar_init(&empty[s], 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, 32 * RT_EPI_WARPS);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < RT_N) cmax[threadIdx.x] = 0ull;
  if (warp == RT_MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                 "r"(RT_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  auto fail = [&](int where) {
    *abort_flag = 1;
    set_status(st, EBV_ERR_TIMEOUT, where);
  };

  if (warp >= RT_CONV_WARP0) {
    // ---- converters: 4 threads per row, 8 columns each (RT_JOBS rows per thread).
    // Thread 0 also issues the stage's X-plane TMA once the stage is free.
    const int ct = threadIdx.x - 32 * RT_CONV_WARP0;
    const int grp = ct & 3;
    int rows[RT_JOBS], fmax[RT_JOBS];
    bool rok[RT_JOBS];
#pragma unroll
    for (int u = 0; u < RT_JOBS; ++u) {
      rows[u] = (ct >> 2) + (RT_CONV_THREADS / 4) * u;
      rok[u] = r0 + rows[u] < n;
      fmax[u] = rok[u] ? rexp[r0 + rows[u]] : 0;
      if (fmax[u] >= kNonFinite) rok[u] = false;  // the epilogue reports NaN for this row
    }
    auto fetch = [&](int sti, double (&v)[RT_JOBS][8]) {
      const int64_t k0 = (int64_t)sti * RT_K + grp * 8;
#pragma unroll
      for (int u = 0; u < RT_JOBS; ++u) {
        const double *src = A + (r0 + rows[u]) * lda + k0;
        if (vec && rok[u] && k0 + 8 <= n) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const double2 t = reinterpret_cast<const double2 *>(src)[j];
            v[u][2 * j] = t.x;
            v[u][2 * j + 1] = t.y;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) v[u][j] = (rok[u] && k0 + j < n) ? src[j] : 0.0;
        }
      }
    };
    double cur[RT_JOBS][8];
    fetch(0, cur);
    for (int sti = 0; sti < nst; ++sti) {
      const int s = sti % RT_STAGES, u = sti / RT_STAGES;
      double nxt[RT_JOBS][8];
      if (sti + 1 < nst) fetch(sti + 1, nxt);
      if (u > 0 && !mbar_wait(&empty[s], (u - 1) & 1, abort_flag)) {
        fail(11);
        break;
      }
      if (ct == 0) {
        mbar_expect_tx(&full[s], RT_S * RT_XPLANE);
        const int y = cb * RT_S * RT_N;
        tma_load_2d(x_plane(s, 0), &tmX, &full[s], sti * RT_K, y);
        tma_load_2d(x_plane(s, RT_S / 2), &tmX, &full[s], sti * RT_K, y + (RT_S / 2) * RT_N);
      }
#pragma unroll
      for (int w = 0; w < RT_JOBS; ++w) {
        long long qb[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) qb[j] = fixed59(cur[w][j], fmax[w]) + kDigitBias;
        const uint32_t off = sw64_offset(rows[w], grp);
#pragma unroll
        for (int p = 0; p < RT_S; ++p) {
          float d[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) d[j] = digit_of(qb[j], p);
          uint4 v;
          v.x = pack_bf16x2(d[0], d[1]);
          v.y = pack_bf16x2(d[2], d[3]);
          v.z = pack_bf16x2(d[4], d[5]);
          v.w = pack_bf16x2(d[6], d[7]);
          *reinterpret_cast<uint4 *>(a_plane(s, p) + off) = v;
        }
      }
      fence_proxy_async_smem();
      mbar_arrive(&full[s]);
      if (sti + 1 < nst) {
#pragma unroll
        for (int w = 0; w < RT_JOBS; ++w)
#pragma unroll
          for (int j = 0; j < 8; ++j) cur[w][j] = nxt[w][j];
      }
    }
    // The X copies this thread issued must land before the CTA may exit.
    if (ct == 0)
      for (int sti = nst - RT_STAGES > 0 ? nst - RT_STAGES : 0; sti < nst; ++sti)
        if (!mbar_wait(&full[sti % RT_STAGES], (sti / RT_STAGES) & 1, nullptr)) set_status(st, EBV_ERR_TIMEOUT, 15);
  } else if (warp == RT_MMA_WARP) {
    if (lane == 0) {
      // ---- MMA issue: per stage and 16-column step, the 55 digit pairs ----
      // bf16 x bf16 -> FP32, both K-major, M = 128, N = nn.
      auto idesc = [](int nn) {
        return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(nn >> 3) << 17) | ((uint32_t)(RT_M >> 4) << 24);
      };
      int committed = -1;
      for (int sti = 0; sti < nst; ++sti) {
        const int s = sti % RT_STAGES, u = sti / RT_STAGES;
        const int sc = sti % SPC, chunk = sti / SPC;
        if (sc == 0 && chunk > 0 && !mbar_wait(tempty, (chunk - 1) & 1, abort_flag)) {
          fail(12);
          break;
        }
        if (!mbar_wait(&full[s], u & 1, abort_flag)) {
          fail(13);
          break;
        }
        tc_fence_after();
        const uint32_t a0 = smem_u32(a_plane(s, 0)), x0 = smem_u32(x_plane(s, 0));
        // For A digit s, the X digits t = 0 .. RT_D-1-s are consecutive 32-row
        // planes and their diagonals d = s + t consecutive 32-column TMEM
        // blocks, so one MMA with N = 32 (RT_D - s) (split at N = 256) covers
        // all pairs (s, t): A is read from shared memory once per digit.
#pragma unroll
        for (int ks = 0; ks < RT_K / 16; ++ks) {
#pragma unroll
          for (int sa = 0; sa < RT_S; ++sa) {
            const uint64_t ad = sw64_desc(a0 + sa * RT_APLANE) + 2 * ks;
            const uint32_t accum = (sc == 0 && ks == 0 && sa == 0) ? 0u : 1u;
#pragma unroll
            for (int t0 = 0; t0 < RT_D - sa; t0 += 8) {
              const int nt = min(8, RT_D - sa - t0);  // X planes in this MMA
              const uint64_t xd = sw64_desc(x0 + t0 * RT_XPLANE) + 2 * ks;
              umma_f16(tmem + (uint32_t)((sa + t0) * RT_N), ad, xd, idesc(nt * RT_N), accum);
            }
          }
        }
        umma_commit(&empty[s]);
        committed = sti;
        if (sc == SPC - 1 || sti == nst - 1) umma_commit(tfull);
      }
      // Every MMA issued must retire before TMEM is released.
      if (committed >= 0 &&
          !mbar_wait(&empty[committed % RT_STAGES], (committed / RT_STAGES) & 1, nullptr))
        set_status(st, EBV_ERR_TIMEOUT, 16);
    }
    __syncwarp();
  } else {
    // ---- drain / epilogue: TMEM lane quarter q = warp, one row per thread ----
    const int q = warp;
    const int row = q * 32 + lane;
    const int64_t gi = r0 + row;
    // Triple-binary32 accumulators per output, kept in this row's TMEM lane
    // (columns RT_TM_H.., RT_TM_M.., RT_TM_L..): (h, m, l) += v exactly up to
    // the rounding of l.
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
    {
      uint32_t z[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) z[j] = 0u;
#pragma unroll
      for (int h = 0; h < RT_N / 16; ++h) {
        tmem_st16(lane_base + RT_TM_H + 16 * h, z);
        tmem_st16(lane_base + RT_TM_M + 16 * h, z);
        tmem_st16(lane_base + RT_TM_L + 16 * h, z);
      }
    }
    bool ok = true;
    for (int chunk = 0; chunk < nchunk; ++chunk) {
      // tcgen05.ld / st are warp-collective: the whole warp goes on or stops.
      if (!__all_sync(0xffffffffu, mbar_wait(tfull, chunk & 1, abort_flag))) {
        fail(17);
        ok = false;
        break;
      }
      tc_fence_after();
#pragma unroll 1
      for (int h = 0; h < RT_N / 8; ++h) {
        uint32_t hw[8], mw[8], lw[8];
        tmem_ld8(lane_base + RT_TM_H + 8 * h, hw);
        tmem_ld8(lane_base + RT_TM_M + 8 * h, mw);
        tmem_ld8(lane_base + RT_TM_L + 8 * h, lw);
#pragma unroll 1
        for (int d = 0; d < RT_D; ++d) {
          const float sc = __int_as_float((127 - 6 * d) << 23);  // 2^(-6d), exact
          uint32_t r[8];
          tmem_ld8(lane_base + (uint32_t)(d * RT_N + 8 * h), r);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            float s1, e1, t1, e2;
            two_sum_f(__uint_as_float(hw[j]), __uint_as_float(r[j]) * sc, s1, e1);
            two_sum_f(__uint_as_float(mw[j]), e1, t1, e2);
            hw[j] = __float_as_uint(s1);
            mw[j] = __float_as_uint(t1);
            lw[j] = __float_as_uint(__uint_as_float(lw[j]) + e2);
          }
        }
        tmem_st8(lane_base + RT_TM_H + 8 * h, hw);
        tmem_st8(lane_base + RT_TM_M + 8 * h, mw);
        tmem_st8(lane_base + RT_TM_L + 8 * h, lw);
      }
      tc_fence_before();
      mbar_arrive(tempty);
    }
    if (ok) {
      tc_fence_after();
      const int fe = gi < n ? rexp[gi] : 0;
#pragma unroll 1
      for (int h = 0; h < RT_N / 8; ++h) {
        uint32_t hw[8], mw[8], lw[8];
        tmem_ld8(lane_base + RT_TM_H + 8 * h, hw);
        tmem_ld8(lane_base + RT_TM_M + 8 * h, mw);
        tmem_ld8(lane_base + RT_TM_L + 8 * h, lw);
        if (gi >= n) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
        const int c = 8 * h + j;
        const int gc = cb * RT_N + c;
        if (gc < nrhs) {
          const int fc = cexp[gc];
          double rv;
          if (fe >= kNonFinite || fc >= kNonFinite) {
            rv = __longlong_as_double(0x7FF8000000000000LL);  // NaN: A or X not finite
          } else {
            // (A X)_ic = value * 2^(E_i + F_c - 10), E = field - 1022
            const double v =
                (double)__uint_as_float(hw[j]) + ((double)__uint_as_float(mw[j]) + (double)__uint_as_float(lw[j]));
            rv = B[gi * ldb + gc] - times_pow2(v, (fe - 1022) + (fc - 1022) - 10);
          }
          R[gi * ldr + gc] = rv;
          const double m = rv != rv ? rv : fabs(rv);  // NaN orders above every number
          atomicMax(&cmax[c], (unsigned long long)__double_as_longlong(m));
        }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x < RT_N && cb * RT_N + (int)threadIdx.x < nrhs && cmax[threadIdx.x])
    atomicMax(&rmax[cb * RT_N + threadIdx.x], cmax[threadIdx.x]);
  if (warp == RT_MMA_WARP)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(RT_TMEM_COLS) : "memory");
}

struct ResidualTcLayout {
  size_t rexp, cexp, xp, total;
  int64_t npad;
  int nrb;
};
ResidualTcLayout residual_tc_layout(int64_t n, int64_t nrhs) {
  ResidualTcLayout L{};
  L.npad = (n + 63) / 64 * 64;
  L.nrb = (int)((nrhs + RT_N - 1) / RT_N);
  size_t off = 0;
  L.rexp = off; off = align256(off + (size_t)n * 4);
  L.cexp = off; off = align256(off + (size_t)L.nrb * RT_N * 4);
  L.xp = off; off = align256(off + (size_t)RT_S * L.nrb * RT_N * L.npad * 2);
  L.total = off;
  return L;
}

}  // namespace

size_t residual_tc_ws(int64_t n, int64_t nrhs) { return residual_tc_layout(n, nrhs).total; }

ebv_status_t residual_tc(const double *A, int64_t lda, int64_t n, const double *X, int64_t ldx, int64_t nrhs,
                         const double *B, int64_t ldb, double *R, int64_t ldr, unsigned long long *rmax, void *ws,
                         bool rows_ready, DevStatus *st, cudaStream_t s) {
  if (n <= 0 || nrhs <= 0) return EBV_OK;
  if (n > INT32_MAX - RT_CHUNK || nrhs > 65535L * RT_N) return EBV_ERR_UNSUPPORTED;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    attr_err = set_smem(k_residual_tc, RT_SMEM);
    if (attr_err == cudaSuccess) attr_err = set_smem(k_row_expmax, 0);
    if (attr_err == cudaSuccess) attr_err = set_smem(k_col_expmax, 0);
    if (attr_err == cudaSuccess) attr_err = set_smem(k_x_planes, 0);
  });
  if (attr_err != cudaSuccess) return EBV_ERR_CUDA;
  const ResidualTcLayout L = residual_tc_layout(n, nrhs);
  char *w = (char *)ws;
  int *rexp = (int *)(w + L.rexp), *cexp = (int *)(w + L.cexp);
  __nv_bfloat16 *xp = (__nv_bfloat16 *)(w + L.xp);
  CUtensorMap map;
  if (!make_map_bf16(&map, xp, L.npad, (int64_t)RT_S * RT_N * L.nrb, L.npad, RT_K, RT_S / 2 * RT_N, 64))
    return EBV_ERR_UNSUPPORTED;
  if (!rows_ready) {
    k_row_expmax<<<ceil_div(n, 8), 256, 0, s>>>(A, lda, n, rexp);
    EBV_TRY(launch_ok());
  }
  EBV_CU(cudaMemsetAsync(cexp, 0, (size_t)L.nrb * RT_N * 4, s));
  k_col_expmax<<<ceil_div(n, 256), 256, 0, s>>>(X, ldx, n, (int)nrhs, cexp);
  EBV_TRY(launch_ok());
  const int gp = (int)std::min<int64_t>(4096, std::max<int64_t>(1, (L.npad * L.nrb * RT_N + 255) / 256));
  k_x_planes<<<gp, 256, 0, s>>>(X, ldx, n, L.npad, (int)nrhs, L.nrb, cexp, xp);
  EBV_TRY(launch_ok());
  prof::Scope ps(s, prof::kResidual, 2.0 * n * n * nrhs);
  dim3 grid(ceil_div(n, RT_M), L.nrb);
  const int vec = (lda % 2 == 0) && ((uintptr_t)A % 16 == 0);  // 16-byte loads of A rows
  k_residual_tc<<<grid, RT_THREADS, RT_SMEM, s>>>(map, A, lda, n, (int)nrhs, rexp, cexp, B, ldb, R, ldr, rmax, vec,
                                                  st);
  return launch_ok();
}

}  // namespace ebv
