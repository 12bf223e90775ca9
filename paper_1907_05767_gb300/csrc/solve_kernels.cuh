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
template <typename T, int NB>
__global__ void __launch_bounds__(4 * NB) k_diag_inverses(MatView<T> F, int64_t n, T *dinv) {
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
// Block substitution in one cooperative launch per triangle (Eq. 1: LY = B,
// then UX = Y), left-looking.  Steps t = 0..nblk-1 visit the row blocks in
// solve order (increasing for L, decreasing for U); each chunk of RC
// right-hand sides is an independent chain of CTAs.  CTA h of a chain owns
// the steps t = h (mod G) and takes them in order: for its block t it folds
// the published blocks s < t into a register accumulator, acc -= F(t,s) X_s,
// in the order they were published, then X_t = D_t^{-1} acc (a tile product
// with the diagonal-block inverse) and releases flag t.  Only the owner ever
// touches block t of B, nothing is written back between folds, and a CTA
// never works on a later block while its current one could advance, so the
// critical path per step is: flag t-1 seen -> X_{t-1} read from L2 -> one
// 64 x 64 x RC fold -> one 64 x 64 x RC solve -> store + release.  The next
// factor tile is fetched into registers while the current fold runs (and
// while the CTA waits).  Every wait is bounded and gives up once the
// workspace status reports an error.  All CTAs must be co-resident: the driver
// launches at most the occupancy limit, cooperatively.
// Dynamic shared memory: trsvl_smem_bytes<T, NB, RC>().
// ---------------------------------------------------------------------------
template <typename T, int NB>
__host__ __device__ constexpr int trsvl_stride() { return NB + 16 / (int)sizeof(T); }  // 16-byte rows

template <typename T, int NB, int RC>
constexpr size_t trsvl_smem_bytes() {
  return sizeof(T) * (2 * (size_t)NB * trsvl_stride<T, NB>() + 2 * (size_t)NB * (RC + 1));
}

template <typename T, int NB, int RC, bool UPPER>
__global__ void __launch_bounds__(256)
    k_trsv_left(MatView<T> F, int64_t n, T *B, int64_t ldb, int nrhs, const T *dinv, int *flags, DevStatus *st) {
  constexpr int NT = 256, FS = trsvl_stride<T, NB>();
  constexpr int PASS = NT / RC, OPT = NB / PASS, LPT = NB * NB / NT;
  static_assert(NT % RC == 0 && NB % PASS == 0 && (NB * NB) % NT == 0, "shape");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T(*Fb)[FS] = reinterpret_cast<T(*)[FS]>(smem_raw);                               // F(t, s)
  T(*Di)[FS] = reinterpret_cast<T(*)[FS]>(smem_raw + sizeof(T) * NB * FS);         // D_t^{-1}
  T(*Xs)[RC + 1] = reinterpret_cast<T(*)[RC + 1]>(smem_raw + 2 * sizeof(T) * NB * FS);  // X_s
  T(*Ac)[RC + 1] = reinterpret_cast<T(*)[RC + 1]>(smem_raw + sizeof(T) * (2 * NB * FS + NB * (RC + 1)));
  __shared__ int s_ok;
  if (st && st->done) return;  // refinement already converged
  const int nblk = ceil_div(n, NB);
  const int nchunk = ceil_div(nrhs, RC);
  const int chunk = blockIdx.x % nchunk, h = blockIdx.x / nchunk;
  const int G = gridDim.x / nchunk;
  if (h >= G) return;
  const int c0 = chunk * RC, wc = min(RC, nrhs - c0);
  int *fl = flags + (int64_t)chunk * nblk;
  auto blk = [&](int s) { return UPPER ? nblk - 1 - s : s; };
  // Blocks s >= t - reach couple into block t (a band limits reach).
  const int reach = (int)max64(1, min64((UPPER ? F.ku + NB - 1 : F.kl + NB - 1) / NB, (int64_t)nblk));
  const int tc = threadIdx.x % RC, tr = threadIdx.x / RC;

  T fr[LPT];  // factor tile in flight
  auto fetch_f = [&](int t, int s) {
    const int64_t i0 = (int64_t)blk(t) * NB, j0 = (int64_t)blk(s) * NB;
    const int hi = (int)min64(NB, n - i0), hj = (int)min64(NB, n - j0);
#pragma unroll
    for (int q = 0; q < LPT; ++q) {
      const int e = threadIdx.x + NT * q, r = e / NB, k = e % NB;
      fr[q] = (r < hi && k < hj) ? F.get(i0 + r, j0 + k) : T(0);
    }
  };

  for (int t = h; t < nblk; t += G) {
    const int64_t i0 = (int64_t)blk(t) * NB;
    const int hi = (int)min64(NB, n - i0);
    const int sb = max(0, t - reach);
    T acc[OPT];
#pragma unroll
    for (int q = 0; q < OPT; ++q) {
      const int r = tr + PASS * q;
      acc[q] = (r < hi && tc < wc) ? B[(i0 + r) * ldb + c0 + tc] : T(0);
    }
    const T *slot = dinv + (int64_t)blk(t) * 4 * NB * NB;
    const T *gmat = slot + (UPPER ? 3 : 2) * NB * NB;  // D_t^{-1} F(t, t-1)
    auto fetch_g = [&]() {
#pragma unroll
      for (int q = 0; q < LPT; ++q) fr[q] = gmat[threadIdx.x + NT * q];
    };
    stage_tile<NB, NT, FS>(&Di[0][0], [&](int r, int k) { return slot[(UPPER ? NB * NB : 0) + r * NB + k]; });
    // Blocks s < t-1 are folded here; block t-1 goes through D_t^{-1} F(t, t-1).
    if (sb < t - 1) fetch_f(t, sb);
    else if (t >= 1) fetch_g();
    for (int s = sb; s < t - 1; ++s) {
      if (threadIdx.x == 0) s_ok = bounded_wait_geq(&fl[s], 1, st, kSpinLimit, s);
      __syncthreads();  // flag seen; the previous fold is done with Fb and Xs
      if (!s_ok) return;
#pragma unroll
      for (int q = 0; q < LPT; ++q) {
        const int e = threadIdx.x + NT * q;
        Fb[e / NB][e % NB] = fr[q];
      }
      {
        const int64_t j0 = (int64_t)blk(s) * NB;
        const int hj = (int)min64(NB, n - j0);
        for (int k = tr; k < NB; k += PASS)
          Xs[k][tc] = (k < hj && tc < wc) ? __ldcg(&B[(j0 + k) * ldb + c0 + tc]) : T(0);
      }
      if (s + 1 < t - 1) fetch_f(t, s + 1);
      else fetch_g();
      __syncthreads();
#pragma unroll 16
      for (int k = 0; k < NB; ++k) {
        const T xk = Xs[k][tc];
#pragma unroll
        for (int q = 0; q < OPT; ++q) acc[q] -= Fb[tr + PASS * q][k] * xk;
      }
    }
    // y = D_t^{-1} acc, before block t-1 is needed.  (Di and Ac are free: the
    // previous block ended with a barrier after its last use of them.)
#pragma unroll
    for (int q = 0; q < OPT; ++q) Ac[tr + PASS * q][tc] = acc[q];
    __syncthreads();
    T y[OPT];
#pragma unroll
    for (int q = 0; q < OPT; ++q) {
      const int r = tr + PASS * q;
      T x = T(0);
#pragma unroll 16
      for (int k = 0; k < NB; ++k) x += Di[r][k] * Ac[k][tc];
      y[q] = x;
    }
    if (t >= 1) {  // x_t = y - (D_t^{-1} F(t, t-1)) x_{t-1}
      if (threadIdx.x == 0) s_ok = bounded_wait_geq(&fl[t - 1], 1, st, kSpinLimit, t - 1);
      __syncthreads();
      if (!s_ok) return;
#pragma unroll
      for (int q = 0; q < LPT; ++q) {
        const int e = threadIdx.x + NT * q;
        Fb[e / NB][e % NB] = fr[q];
      }
      {
        const int64_t j0 = (int64_t)blk(t - 1) * NB;
        const int hj = (int)min64(NB, n - j0);
        for (int k = tr; k < NB; k += PASS)
          Xs[k][tc] = (k < hj && tc < wc) ? __ldcg(&B[(j0 + k) * ldb + c0 + tc]) : T(0);
      }
      __syncthreads();
#pragma unroll 16
      for (int k = 0; k < NB; ++k) {
        const T xk = Xs[k][tc];
#pragma unroll
        for (int q = 0; q < OPT; ++q) y[q] -= Fb[tr + PASS * q][k] * xk;
      }
    }
#pragma unroll
    for (int q = 0; q < OPT; ++q) {
      const int r = tr + PASS * q;
      if (r < hi && tc < wc) B[(i0 + r) * ldb + c0 + tc] = y[q];
    }
    // The barrier orders every thread's stores of x_t before thread 0's
    // gpu-scope fence, which makes them visible before the flag (cumulativity).
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      st_release(&fl[t], 1);
    }
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
