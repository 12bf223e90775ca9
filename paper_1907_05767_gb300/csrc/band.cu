// Banded factorisation and solve (the sparse case of the paper's first
// experiment, stored as a band).  Without row exchanges the L vectors of step
// r reach rows r+1..r+kl only and the U vectors columns r+1..r+ku only, so all
// fill-in stays inside the band (Eq. 6a-c restricted to the band).
//
// Right-looking over 64-column leaf blocks: per block, the equal
// bi-vectorised diagonal kernel, L21 for the <= kl rows below, U12 for the
// <= ku columns to the right, and one dense (kl x ku x 64) window update.  All
// kernels read through a band view (out-of-band entries read as 0, never
// written).
//
// Variable band (the profile, or skyline, of the matrix): a first kernel finds
// each 64-block's envelope -- the first non-zero left of the diagonal over the
// block's rows, above it over its columns -- and the L21, U12 and update CTAs
// whose block lies outside it for the current panel return at once, so a band
// whose width varies costs the work of its envelope, not of its widest row.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include "internal.h"
#include "solve_driver.cuh"

namespace ebv {

namespace {

template <typename T>
struct BandGemm;
template <>
struct BandGemm<double> {
  static constexpr int BM = 32, BN = 32, BK = 16, TM = 2, TN = 2;
};
// FP64 windows of fewer than four 32 x 32 tiles per SM (a band's): 16 x 16
// tiles, one output per thread.  An FP64 warp instruction costs the pipe the
// same whatever the tile, so the DFMA time is fixed and the small tiles only
// balance the SMs (a 512 x 512 window: 1024 tiles over 152 SMs against 256 of
// 32 x 32, two per SM on most and one on the rest; 512 x 512 Laplacian
// 649 -> 621 ms).  Wide windows (dense symmetric) keep 32 x 32: there the
// extra shared-memory loads of the small tiles cost more (1320 -> 1371 ms).
struct BandGemmNarrow {
  static constexpr int BM = 16, BN = 16, BK = 16, TM = 1, TN = 1;
};
template <>
struct BandGemm<float> {
  static constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
};

// Block envelope (see Envelope): one warp per index i scans row i left of the
// diagonal from its band edge for the first non-zero and column i above the
// diagonal from its band edge likewise, and lowers lo[i/64] / up[i/64] to
// what it found (i itself when the part is empty).  lo and up start above any
// index.  The column scan reads one element per row (stride ld) but stops at
// the first non-zero, which for a band matrix is near the band edge.
template <typename T, bool XV>
__global__ void __launch_bounds__(256) k_band_envelope(MatView<T, XV> A, int64_t n, int32_t *lo, int32_t *up) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * 8 + threadIdx.x / 32;
  if (i >= n) return;
  int64_t first = i;
  for (int64_t j0 = max64(0, i - A.kl); j0 < i; j0 += 32) {  // row i, columns j0 .. i-1
    const int64_t j = j0 + lane;
    const unsigned nz = __ballot_sync(0xffffffffu, j < i && A.get(i, j) != T(0));
    if (nz) {
      first = j0 + __ffs(nz) - 1;
      break;
    }
  }
  if (lane == 0) atomicMin(&lo[i / 64], (int32_t)first);
  first = i;
  for (int64_t r0 = max64(0, i - A.ku); r0 < i; r0 += 32) {  // column i, rows r0 .. i-1
    const int64_t r = r0 + lane;
    const unsigned nz = __ballot_sync(0xffffffffu, r < i && A.get(r, i) != T(0));
    if (nz) {
      first = r0 + __ffs(nz) - 1;
      break;
    }
  }
  if (lane == 0) atomicMin(&up[i / 64], (int32_t)first);
}

// L21 = A21 U11^{-1} by substitution (FP64 panels): one warp per row of
// A21, NW rows per CTA; lane l holds columns l and l+32 of the row.  Step j: the lane holding
// column j forms l_ij = (a_ij - sum_{k<j} l_ik u_kj) / u_jj with the FP64
// reciprocal and passes it by shuffle; every lane subtracts l_ij u_jc from
// its later columns c (U11 and the reciprocals staged in shared memory).  The
// 64-step chain per row needs no inverse of U11, so the diagonal-block kernel
// only factors; rows run on many SMs.  Rows of 64-blocks outside the
// envelope hold zeros and are skipped.
template <typename T, int NB, int NW, bool XV>
__global__ void __launch_bounds__(32 * NW) k_trsm_ru_subst(MatView<T, XV> A, int64_t c0, int w, int64_t rb,
                                                           int64_t re, Envelope env) {
  constexpr int NT = 32 * NW;
  __shared__ T Us[NB][NB + 1];
  __shared__ T rc[NB];
  for (int e = threadIdx.x; e < NB * NB; e += NT) {
    const int k = e / NB, c = e % NB;
    Us[k][c] = (k < w && c < w && c >= k) ? A.get(c0 + k, c0 + c) : T(0);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < NB; k += NT) rc[k] = k < w ? pivot_rcp(Us[k][k]) : T(0);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t i = rb + (int64_t)blockIdx.x * NW + (threadIdx.x >> 5);
  if (i >= re || env.rows_empty(i, c0 + w)) return;
  T a0 = lane < w ? A.get(i, c0 + lane) : T(0);
  T a1 = lane + 32 < w ? A.get(i, c0 + lane + 32) : T(0);
  for (int j = 0; j < w; ++j) {
    const T mine = j < 32 ? a0 : a1;
    const T l = __shfl_sync(0xffffffffu, mine, j & 31) * rc[j];  // Eq. 6a
    if (lane == (j & 31)) {
      if (j < 32) a0 = l;
      else a1 = l;
    }
    if (lane > j) a0 -= l * Us[j][lane];
    if (lane + 32 > j) a1 -= l * Us[j][lane + 32];
  }
  if (lane < w) A.put(i, c0 + lane, a0);
  if (lane + 32 < w) A.put(i, c0 + lane + 32, a1);
}

// U12 = L11^{-1} A12 by substitution (FP64 panels): one warp per column of
// A12 (8 per CTA, the 64 x 8 block staged with whole rows); lane l holds rows
// l and l+32.  Step k: u_kj is final; it goes by shuffle to every lane,
// which subtracts l_rk u_kj from its later rows r (Eq. 6b; L11 unit lower).
template <typename T, int NB, bool XV>
__global__ void __launch_bounds__(256) k_trsm_ll_subst(MatView<T, XV> A, int64_t c0, int w, int64_t cb, int64_t ce,
                                                       Envelope env) {
  __shared__ T Ls[NB][NB + 1];
  __shared__ T Bs[NB][8 + 1];
  const int64_t j0 = cb + (int64_t)blockIdx.x * 8;
  if (env.cols_empty(j0, c0 + w) && env.cols_empty(min64(ce - 1, j0 + 7), c0 + w)) return;
  for (int e = threadIdx.x; e < NB * NB; e += 256) {
    const int r = e / NB, k = e % NB;
    Ls[r][k] = (r < w && k < r) ? A.get(c0 + r, c0 + k) : T(0);
  }
  for (int e = threadIdx.x; e < NB * 8; e += 256) {
    const int r = e / 8, c = e % 8;
    Bs[r][c] = (r < w && j0 + c < ce) ? A.get(c0 + r, j0 + c) : T(0);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, cw = threadIdx.x >> 5;
  if (j0 + cw < ce) {
    T b0 = Bs[lane][cw], b1 = Bs[lane + 32][cw];
    for (int k = 0; k < w; ++k) {
      const T u = __shfl_sync(0xffffffffu, k < 32 ? b0 : b1, k & 31);
      if (lane > k) b0 -= Ls[lane][k] * u;
      if (lane + 32 > k) b1 -= Ls[lane + 32][k] * u;
    }
    Bs[lane][cw] = b0;
    Bs[lane + 32][cw] = b1;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NB * 8; e += 256) {
    const int r = e / 8, c = e % 8;
    if (r < w && j0 + c < ce) A.put(c0 + r, j0 + c, Bs[r][c]);
  }
}

// Side streams and events of the FP64 panels' overlaps, one set per device,
// made by the first factorisation on the device: `side` takes the
// look-ahead's trailing updates, `side2` each panel's U12 (concurrent with
// its L21).
struct BandPipe {
  cudaStream_t side = nullptr, side2 = nullptr;
  cudaEvent_t fork = nullptr, go = nullptr, join = nullptr, join2 = nullptr, dg = nullptr, u12 = nullptr,
              done[2] = {};
  bool ready = false;
};
constexpr int kMaxPipeDevices = 64;
BandPipe g_band_pipe[kMaxPipeDevices];
std::mutex g_band_pipe_mutex;

ebv_status_t band_pipe(BandPipe **out) {
  int dev = 0;
  EBV_CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxPipeDevices) return EBV_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_band_pipe_mutex);
  BandPipe &p = g_band_pipe[dev];
  if (!p.ready) {
    EBV_CU(cudaStreamCreateWithFlags(&p.side, cudaStreamNonBlocking));
    EBV_CU(cudaStreamCreateWithFlags(&p.side2, cudaStreamNonBlocking));
    for (cudaEvent_t *e : {&p.fork, &p.go, &p.join, &p.join2, &p.dg, &p.u12, &p.done[0], &p.done[1]})
      EBV_CU(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    p.ready = true;
  }
  *out = &p;
  return EBV_OK;
}

bool g_band_envelope = true;  // testing hook: false = every CTA of the band window works
// FP64 panels' overlaps (testing hook): 0 = serial; 1 = look-ahead for the
// symmetric storages, U12 beside L21 for the general ones; 2 (default) = also
// look-ahead for the general band (with the 16 x 16 window tiles: 512 x 512
// Laplacian 620 -> 603 ms, the disc's variable band 650 -> 621 ms).
int g_band_overlap = 2;
bool g_band_subst = true;     // FP64 panels: substitution L21 / U12 (true) or inverse tile products
// FP64 panels' diagonal blocks: the register-resident kernel (true) or the
// blocked 16 x 16 sub-block kernel (testing hook)
bool g_diag_lu = true;
// Band panels: the diagonal block on one CTA with L21 / U12 as separate
// launches (false, every storage) or one thread-block-cluster launch per
// panel (true, a testing hook).  Measured on the 512 x 512 Laplacian, factor
// + solve: 565 ms against 1147 ms on clusters.
bool g_band_cluster = false;

// Symmetric band with both halves stored (EBV_BAND_SYM): the factorisation
// runs on the lower half only (the lower-half view of the same array), then
// this fills the upper half with U = D L^T, u_ij = d_i l_ji (Eq. 6a-b scale
// both vectors by the same pivot), the one product the per-panel U12 kernel
// formed.  One thread per stored entry i, j = i+1 .. i+kl; the writes of a
// row are contiguous.
template <typename T>
__global__ void __launch_bounds__(256) k_band_fill_upper(T *ab, int64_t ldab, int64_t n, int64_t kl) {
  const int64_t total = n * kl;
  for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < total; e += (int64_t)gridDim.x * 256) {
    const int64_t i = e / kl, t = e % kl + 1, j = i + t;
    if (j < n) ab[i * ldab + kl + t] = ab[i * ldab + kl] * ab[j * ldab + kl - t];
  }
}

// Binary32 working copy of the whole band array (mixed precisions): count
// elements, grid-stride.  Slots outside the matrix are copied too and, as in
// the FP64 array, never read.
__global__ void __launch_bounds__(256) k_band_narrow(const double *ab, float *lo, int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < count; e += (int64_t)gridDim.x * 256)
    lo[e] = (float)ab[e];
}

// Profile (skyline) storage, EBV_PROFILE: per 64-block header of int32
// lo[nb], int32 up[nb], int64 offL[nb], int64 offU[nb] (nb = ceil(n/64)),
// then the values from byte profile_header_bytes(n) (see MatView).
size_t profile_header_bytes(int64_t n) { return align256((size_t)24 * (size_t)ceil_div(n, kNB)); }

template <typename T>
XView<T> profile_view(void *buf, int64_t n, int64_t kl, int64_t ku) {
  const int64_t nb = ceil_div(n, kNB);
  char *h = (char *)buf;
  XView<T> v{(T *)(h + profile_header_bytes(n)), 0, kl, ku};
  v.plo = (const int32_t *)h;
  v.pup = (const int32_t *)(h + 4 * nb);
  v.poffL = (const int64_t *)(h + 8 * nb);
  v.poffU = (const int64_t *)(h + 16 * nb);
  return v;
}

template <typename T, bool XV>
ebv_status_t band_factor_t(MatView<T, XV> A, int64_t n, int32_t *info, T *inv, int32_t *env_lo, bool sym, T *bcast,
                           cudaStream_t s, bool envelope = true) {
  const Shadow<float> none{nullptr, nullptr, 0, nullptr};
  using G = BandGemm<T>;
  EBV_TRY((prepare_leaf_kernels<T, float>()));
  if constexpr (XV) EBV_TRY(prepare_xview_kernels<T>());
  constexpr size_t smem = pair_smem_bytes<T, kNB>();
  Envelope env;
  if (A.plo) {  // profile storage: the stored extents are the block envelope
    if (g_band_envelope) {
      env.lo = A.plo;
      env.up = A.pup;
    }
  } else if (g_band_envelope && envelope) {
    const int64_t nblk = ceil_div(n, kNB);
    int32_t *env_up = env_lo + nblk;
    EBV_CU(cudaMemsetAsync(env_lo, 0x7f, 2 * nblk * sizeof(int32_t), s));  // 0x7f7f7f7f > any index
    prof::Scope ps(s, prof::kOther, 0.0);
    k_band_envelope<T><<<ceil_div(n, 8), 256, 0, s>>>(A, n, env_lo, env_up);
    EBV_TRY(launch_ok());
    env.lo = env_lo;
    env.up = env_up;
  }
  // Panels on a thread-block cluster (diagonal block, L21 and U12 in one
  // launch) only when the testing hook asks for them, for the band views
  // (not the profile or dense views).
  bool cluster = !A.plo && A.kl < kDenseBand && g_band_cluster && cluster_panel_enabled() &&
                 cluster_panel_fits(sizeof(T) == 8, kNB, std::min<int64_t>(n, kNB + A.kl), sym ? 0 : A.ku);
  // The diagonal-block kernel reads its still unfactored block; in the
  // lower-half symmetric storage that view reads a_ji above the diagonal.
  MatView<T, XV> Araw = A;
  Araw.symraw = true;
  static const int sm_count = [] {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 0;
    return sms;
  }();
  // FP64 look-ahead for the symmetric storages (whose trailing updates, the
  // block-lower half only, leave the diagonal block's SM its FP64 units;
  // 512 x 512 Laplacian 638 -> 577 ms) and the general band (620 -> 603 ms;
  // g_band_overlap).  General bands: each panel's U12 on a second side
  // stream, concurrent with its L21 (both read only the diagonal block and
  // their own entries).  The side streams fork from `s` here and `s` waits
  // for them at the end.
  const bool fp64_subst = sizeof(T) == 8 && g_band_subst && !cluster;
  // (Four panels or fewer, the small dense systems: the general look-ahead's
  // events cost more than it hides, n = 256 0.522 -> 0.529 ms.)
  const bool ahead = fp64_subst && n > 2 * kNB && (sym ? g_band_overlap >= 1 : g_band_overlap >= 2 && n > 4 * kNB);
  const bool u12_side = fp64_subst && !sym && n > kNB && g_band_overlap >= 1;
  BandPipe *pipe = nullptr, *bp = nullptr;
  if (ahead || u12_side) {
    EBV_TRY(band_pipe(&bp));
    EBV_CU(cudaEventRecord(bp->fork, s));
    if (ahead) EBV_CU(cudaStreamWaitEvent(bp->side, bp->fork, 0));
    if (u12_side) EBV_CU(cudaStreamWaitEvent(bp->side2, bp->fork, 0));
    if (ahead) pipe = bp;
  }
  for (int64_t c0 = 0; c0 < n; c0 += kNB) {
    const int w = (int)std::min<int64_t>(kNB, n - c0);
    const int64_t rb = c0 + w, re = std::min<int64_t>(n, c0 + w + A.kl);
    const int64_t cb = c0 + w, ce = std::min<int64_t>(n, c0 + w + A.ku);
    if (cluster) {
      const ebv_status_t st = cluster_panel(sizeof(T) == 8, A.base, A.ld, A.kl, A.ku, A.symlo, c0, w, re - c0,
                                            sym ? 0 : ce - cb, info, bcast, s);
      if (st == EBV_ERR_UNSUPPORTED && c0 == 0 && !A.symlo) {
        cluster = false;  // the device cannot run the cluster: one-CTA kernels from here on
      } else {
        EBV_TRY(st);
        // (symmetric storages: U12 = D11 L21^T is implied, the lower-half view reads it so)
        if (re > rb && ce > cb) {
          prof::Scope ps(s, prof::kSimtGemm, 2.0 * (re - rb) * (ce - cb) * w);
          dim3 grid(ceil_div(ce - cb, G::BN), ceil_div(re - rb, G::BM));
          k_gemm_nn<T, G::BM, G::BN, G::BK, G::TM, G::TN>
              <<<grid, (G::BM / G::TM) * (G::BN / G::TN), 0, s>>>(A, rb, cb, c0, re - rb, ce - cb, w, sym ? 1 : 0,
                                                                  env);
          EBV_TRY(launch_ok());
        }
        continue;
      }
    }
    if constexpr (sizeof(T) == 8) {
      if (g_band_subst) {
        // FP64: the diagonal block factored alone (no inverses: two thirds
        // of its FP64 work), then L21 and U12 by substitution over many SMs.
        // Look-ahead: the trailing update is split into
        // the next panel's 64 columns (on `s`, the critical path) and the
        // rest (on the side stream, overlapping the next diagonal block,
        // which runs on one SM).  Panel p's diagonal block and L21 wait for
        // the rest-update of panel p-2, its U12 for that of panel p-1 (the
        // only ones touching those entries).
        const int64_t p = c0 / kNB;
        if (pipe && p >= 2) EBV_CU(cudaStreamWaitEvent(s, pipe->done[p & 1], 0));
        {
          prof::Scope ps(s, prof::kPanel, 2.0 * w * w * w / 3.0);
          if (g_diag_lu)
            k_diag_lu<T><<<1, 256, 0, s>>>(Araw, c0, w, info);
          else
            k_diag_factor<T, kNB, 4 * kNB, XV, false>
                <<<1, 4 * kNB, diagb_smem_bytes<T, kNB>(), s>>>(Araw, c0, w, info, nullptr);
          EBV_TRY(launch_ok());
        }
        const bool u12_beside = u12_side && ce > cb;
        if (u12_beside) {  // U12 on side2 after the diagonal block (and the rest-update of panel p-1)
          EBV_CU(cudaEventRecord(bp->dg, s));
          EBV_CU(cudaStreamWaitEvent(bp->side2, bp->dg, 0));
          if (pipe && p >= 1) EBV_CU(cudaStreamWaitEvent(bp->side2, pipe->done[(p - 1) & 1], 0));
          prof::Scope ps(bp->side2, prof::kTrsm, 1.0 * w * w * (ce - cb));
          k_trsm_ll_subst<T, kNB><<<ceil_div(ce - cb, 8), 256, 0, bp->side2>>>(A, c0, w, cb, ce, env);
          EBV_TRY(launch_ok());
          EBV_CU(cudaEventRecord(bp->u12, bp->side2));
        }
        if (re > rb) {
          prof::Scope ps(s, prof::kL21, 1.0 * (re - rb) * w * w);
          // Symmetric storages: four rows per CTA, so one warp per SMSP keeps
          // its FP64 pipe to itself (each row's chain issues three FP64 warp
          // instructions per step; 512 x 512 Laplacian 621 -> 602 ms).  The
          // general band keeps eight: its U12 runs beside on other SMs.
          if (sym)
            k_trsm_ru_subst<T, kNB, 4><<<ceil_div(re - rb, 4), 128, 0, s>>>(A, c0, w, rb, re, env);
          else
            k_trsm_ru_subst<T, kNB, 8><<<ceil_div(re - rb, 8), 256, 0, s>>>(A, c0, w, rb, re, env);
          EBV_TRY(launch_ok());
        }
        if (pipe && p >= 1) EBV_CU(cudaStreamWaitEvent(s, pipe->done[(p - 1) & 1], 0));
        // (symmetric storages: U12 = D11 L21^T is implied, the lower-half view reads it so)
        if (u12_beside) {
          EBV_CU(cudaStreamWaitEvent(s, bp->u12, 0));
        } else if (ce > cb && !sym) {
          prof::Scope ps(s, prof::kTrsm, 1.0 * w * w * (ce - cb));
          k_trsm_ll_subst<T, kNB><<<ceil_div(ce - cb, 8), 256, 0, s>>>(A, c0, w, cb, ce, env);
          EBV_TRY(launch_ok());
        }
        if (re > rb && ce > cb) {
          auto gemm = [&](int64_t n0, int64_t n1, cudaStream_t st) -> ebv_status_t {
            if (n1 <= n0) return EBV_OK;
            prof::Scope ps(st, prof::kSimtGemm, 2.0 * (re - rb) * (n1 - n0) * w);
            if constexpr (sizeof(T) == 8) {
              using H = BandGemmNarrow;
              if ((int64_t)ceil_div(n1 - n0, G::BN) * ceil_div(re - rb, G::BM) < 4 * sm_count) {
                dim3 grid(ceil_div(n1 - n0, H::BN), ceil_div(re - rb, H::BM));
                k_gemm_nn<T, H::BM, H::BN, H::BK, H::TM, H::TN>
                    <<<grid, (H::BM / H::TM) * (H::BN / H::TN), 0, st>>>(A, rb, n0, c0, re - rb, n1 - n0, w,
                                                                         sym ? 1 : 0, env);
                return launch_ok();
              }
            }
            constexpr int nt = (G::BM / G::TM) * (G::BN / G::TN);
            dim3 grid(ceil_div(n1 - n0, G::BN), ceil_div(re - rb, G::BM));
            k_gemm_nn<T, G::BM, G::BN, G::BK, G::TM, G::TN><<<grid, nt, 0, st>>>(A, rb, n0, c0, re - rb, n1 - n0, w,
                                                                                    sym ? 1 : 0, env);
            return launch_ok();
          };
          const int64_t split = pipe ? std::min<int64_t>(ce, cb + kNB) : ce;
          EBV_TRY(gemm(cb, split, s));
          if (split < ce) {
            EBV_CU(cudaEventRecord(pipe->go, s));
            EBV_CU(cudaStreamWaitEvent(pipe->side, pipe->go, 0));
            EBV_TRY(gemm(split, ce, pipe->side));
          }
        }
        if (pipe) EBV_CU(cudaEventRecord(pipe->done[p & 1], pipe->side));
        continue;
      }
    }
    {
      prof::Scope ps(s, prof::kPanel, 2.0 * w * w * w / 3.0);
      k_diag_factor<T, kNB, 4 * kNB><<<1, 4 * kNB, diagb_smem_bytes<T, kNB>(), s>>>(Araw, c0, w, info, inv);
      EBV_TRY(launch_ok());
    }
    // FP64: 16-row / 16-column strips, four times the CTAs of one 64 x 64
    // tile each (a band has only kl rows / ku columns per step).
    if (re > rb) {
      prof::Scope ps(s, prof::kL21, 2.0 * (re - rb) * w * w);
      if constexpr (sizeof(T) == 8)
        k_trsm_ru_strip<T, float, kNB, 16><<<ceil_div(re - rb, 16), 256, smem, s>>>(A, c0, w, rb, re, inv, none,
                                                                                      env);
      else
        k_trsm_ru<T, float, kNB><<<ceil_div(re - rb, kNB), 256, smem, s>>>(A, c0, w, rb, re, inv, none, env);
      EBV_TRY(launch_ok());
    }
    // (symmetric storages: U12 = D11 L21^T is implied, the lower-half view reads it so)
    if (ce > cb && !sym) {
      prof::Scope ps(s, prof::kTrsm, 2.0 * w * w * (ce - cb));
      if constexpr (sizeof(T) == 8)
        k_trsm_ll_multi<T, float, kNB, kTrsmMaxBlocks, 16>
            <<<ceil_div(ce - cb, 16), 256, trsm_multi_smem_bytes<T, kNB, kTrsmMaxBlocks>(), s>>>(A, c0, w, cb, ce,
                                                                                               inv, none, env);
      else
        k_trsm_ll<T, float, kNB><<<ceil_div(ce - cb, kNB), 256, smem, s>>>(A, c0, w, cb, ce, inv, none, env);
      EBV_TRY(launch_ok());
    }
    if (re > rb && ce > cb) {
      prof::Scope ps(s, prof::kSimtGemm, 2.0 * (re - rb) * (ce - cb) * w);
      dim3 grid(ceil_div(ce - cb, G::BN), ceil_div(re - rb, G::BM));
      // symmetric: L21 D11 L21^T, only its block-lower part (the diagonal 64-blocks whole)
      k_gemm_nn<T, G::BM, G::BN, G::BK, G::TM, G::TN>
          <<<grid, (G::BM / G::TM) * (G::BN / G::TN), 0, s>>>(A, rb, cb, c0, re - rb, ce - cb, w, sym ? 1 : 0, env);
      EBV_TRY(launch_ok());
    }
  }
  if (pipe) {
    EBV_CU(cudaEventRecord(pipe->join, pipe->side));
    EBV_CU(cudaStreamWaitEvent(s, pipe->join, 0));
  }
  if (u12_side) {
    EBV_CU(cudaEventRecord(bp->join2, bp->side2));
    EBV_CU(cudaStreamWaitEvent(s, bp->join2, 0));
  }
  return EBV_OK;
}

// R = B - A X for a row-band A, multi-word binary32 accumulation as in the
// dense residual.  One warp per row; the lanes stride over the row's band.
// symlo: ab holds the lower half of a symmetric band (ku = kl); a_ij above
// the diagonal is read as a_ji.
__global__ void __launch_bounds__(256)
    k_band_residual_df(const double *ab, int64_t ldab, int64_t n, int64_t kl, int64_t ku, bool symlo,
                       const float *xhi, const float *xlo, int nrhs, const double *B, int64_t ldb, double *R,
                       int64_t ldr, unsigned long long *rmax, const DevStatus *st) {
  if (st && st->done) return;
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (i >= n) return;
  const int64_t j0 = max64(0, i - kl), j1 = min64(n - 1, i + ku);
  for (int c = 0; c < nrhs; ++c) {
    TripleF acc;
    acc.zero();
    for (int64_t j = j0 + lane; j <= j1; j += 32) {
      float a_h, a_l;
      split_f64((symlo && j > i) ? ab[j * ldab + (i - j + kl)] : ab[i * ldab + (j - i + kl)], a_h, a_l);
      acc.fma_split(a_h, a_l, xhi[j * nrhs + c], xlo[j * nrhs + c]);
    }
    // Error-free (up to the l words) warp reduction of the triples.
    for (int off = 16; off > 0; off >>= 1) {
      TripleF o;
      o.h = __shfl_xor_sync(0xffffffffu, acc.h, off);
      o.m = __shfl_xor_sync(0xffffffffu, acc.m, off);
      o.l = __shfl_xor_sync(0xffffffffu, acc.l, off);
      acc.add(o);
    }
    if (lane == 0) {
      const double rv = B[i * ldb + c] - acc.value();
      R[i * ldr + c] = rv;
      atomicMax(&rmax[c], (unsigned long long)__double_as_longlong(fabs(rv)));
    }
  }
}

// R = B - A X through a view (profile storage, the lower triangle of a
// symmetric dense matrix), as k_band_residual_df: one warp per row over the
// view's window, entries outside the profile read 0.
__global__ void __launch_bounds__(256)
    k_view_residual_df(XView<double> A, int64_t n, const float *xhi, const float *xlo, int nrhs, const double *B,
                       int64_t ldb, double *R, int64_t ldr, unsigned long long *rmax, const DevStatus *st) {
  if (st && st->done) return;
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (i >= n) return;
  const int64_t j0 = max64(0, i - A.kl), j1 = min64(n - 1, i + A.ku);
  for (int c = 0; c < nrhs; ++c) {
    TripleF acc;
    acc.zero();
    for (int64_t j = j0 + lane; j <= j1; j += 32) {
      if (!A.in(i, j)) continue;
      float a_h, a_l;
      split_f64(A.raw(i, j), a_h, a_l);
      acc.fma_split(a_h, a_l, xhi[j * nrhs + c], xlo[j * nrhs + c]);
    }
    for (int off = 16; off > 0; off >>= 1) {
      TripleF o;
      o.h = __shfl_xor_sync(0xffffffffu, acc.h, off);
      o.m = __shfl_xor_sync(0xffffffffu, acc.m, off);
      o.l = __shfl_xor_sync(0xffffffffu, acc.l, off);
      acc.add(o);
    }
    if (lane == 0) {
      const double rv = B[i * ldb + c] - acc.value();
      R[i * ldr + c] = rv;
      atomicMax(&rmax[c], (unsigned long long)__double_as_longlong(fabs(rv)));
    }
  }
}

}  // namespace

// Workspace of the banded factorisation: the status block, the inverses of
// the current leaf's two triangular factors (used right after they are made),
// the block envelope (two int32 per 64-block) and the cluster panels' pivot
// column scratch (two slots of 64 + kl + 1 elements).
static size_t band_inv_bytes(ebv_prec_t prec) { return align256((size_t)2 * kNB * kNB * (prec == EBV_FP64 ? 8 : 4)); }
static size_t band_env_bytes(int64_t n) { return align256((size_t)2 * ceil_div(n, kNB) * sizeof(int32_t)); }
static size_t band_bcast_bytes(int64_t kl, ebv_prec_t prec) {
  return align256((size_t)2 * (kNB + kl + 1) * (prec == EBV_FP64 ? 8 : 4));
}
size_t band_factor_ws(int64_t n, int64_t kl, int64_t, ebv_prec_t prec) {
  return kStatusBytes + band_inv_bytes(prec) + band_env_bytes(n) + band_bcast_bytes(kl, prec);
}
void set_band_envelope(bool on) { g_band_envelope = on; }
void set_band_cluster(bool on) { g_band_cluster = on; }
void set_band_overlap(int mode) { g_band_overlap = mode; }
void set_diag_lu(bool on) { g_diag_lu = on; }
size_t band_solve_ws(int64_t n, int64_t nrhs, ebv_prec_t prec) {
  return solve_layout(n, nrhs, prec == EBV_FP64 ? 8 : 4).total;
}

ebv_status_t band_factor(const ebv_desc_t *d, ebv_prec_t prec, void *a, void *lowp, int32_t *info, void *ws,
                         size_t ws_bytes, cudaStream_t s) {
  EBV_CU(cudaMemsetAsync(info, 0, sizeof(int32_t), s));
  if (ws) EBV_CU(cudaMemsetAsync(ws, 0, sizeof(DevStatus), s));
  if (d->n == 0) return EBV_OK;
  if (!ws || ws_bytes < band_factor_ws(d->n, ws_kl(d), d->ku, prec)) return EBV_ERR_WORKSPACE;
  char *inv = (char *)ws + kStatusBytes;
  int32_t *env = (int32_t *)(inv + band_inv_bytes(prec));
  char *bcast = (char *)env + band_env_bytes(d->n);
  const bool lower = d->storage == EBV_BAND_SYM_LOWER;
  const bool sym = d->storage == EBV_BAND_SYM || lower;
  if (d->storage == EBV_DENSE_SYM) {  // the band panels on the lower triangle of a dense array
    if (prec == EBV_FP64)
      return band_factor_t<double>(dense_symlo_view((double *)a, d->ld), d->n, info, (double *)inv, env, true,
                                   (double *)bcast, s);
    if (prec == EBV_FP32)
      return band_factor_t<float>(dense_symlo_view((float *)a, d->ld), d->n, info, (float *)inv, env, true,
                                  (float *)bcast, s);
    return EBV_ERR_UNSUPPORTED;
  }
  if (d->storage == EBV_PROFILE) {
    if (prec == EBV_FP64)
      return band_factor_t<double>(profile_view<double>(a, d->n, d->kl, d->ku), d->n, info, (double *)inv, env,
                                   false, (double *)bcast, s);
    if (prec == EBV_FP32)
      return band_factor_t<float>(profile_view<float>(a, d->n, d->kl, d->ku), d->n, info, (float *)inv, env, false,
                                  (float *)bcast, s);
    return EBV_ERR_UNSUPPORTED;
  }
  // the factorisation in the view of the lower half (both symmetric
  // storages) or of the whole band; EBV_BAND_SYM then gets its upper half
  auto run = [&](auto *p, auto *iv, auto *bc) -> ebv_status_t {
    if (!sym) return band_factor_t(band_view(p, d->ld, d->kl, d->ku), d->n, info, iv, env, false, bc, s);
    EBV_TRY(band_factor_t(symlo_view(p, d->ld, d->kl), d->n, info, iv, env, true, bc, s));
    if (lower || d->kl == 0) return EBV_OK;
    using E = std::remove_pointer_t<decltype(p)>;
    const int64_t total = d->n * d->kl;
    k_band_fill_upper<E><<<(unsigned)std::min<int64_t>(8192, (total + 255) / 256), 256, 0, s>>>(p, d->ld, d->n,
                                                                                               d->kl);
    return launch_ok();
  };
  if (prec == EBV_FP64) return run((double *)a, (double *)inv, (double *)bcast);
  if (prec == EBV_FP32) return run((float *)a, (float *)inv, (float *)bcast);
  if (prec == EBV_MIXED_BF16 || prec == EBV_MIXED_FP16) {
    // FP32 factors of the FP64 band in lowp (same layout); a stays untouched
    // for the refinement's residual.  The band's updates run in FP32 SIMT.
    const int64_t count = d->n * d->ld;
    k_band_narrow<<<(unsigned)std::min<int64_t>(4096, (count + 255) / 256), 256, 0, s>>>((const double *)a,
                                                                                         (float *)lowp, count);
    EBV_TRY(launch_ok());
    return run((float *)lowp, (float *)inv, (float *)bcast);
  }
  return EBV_ERR_UNSUPPORTED;
}

ebv_status_t band_solve(const ebv_desc_t *d, ebv_prec_t prec, const void *lu, const double *a_orig, void *b,
                        int64_t nrhs, int64_t ldb, const ebv_refine_t *refine, ebv_refine_report_t *rep, void *ws,
                        size_t ws_bytes, cudaStream_t s) {
  const int64_t n = d->n;
  const bool fp64 = prec == EBV_FP64;
  const bool lower = d->storage == EBV_BAND_SYM_LOWER;
  const DenseSolveLayout L = solve_layout(n, nrhs, fp64 ? 8 : 4);
  if (!ws || ws_bytes < L.total) return EBV_ERR_WORKSPACE;
  EBV_CU(cudaMemsetAsync(ws, 0, sizeof(DevStatus), s));
  if (n == 0 || nrhs == 0) return EBV_OK;
  auto residual = [&](const double *x, int64_t ldx, float *xhi, float *xlo, const double *bs, double *r,
                      unsigned long long *rmax, DevStatus *st, bool) -> ebv_status_t {
    k_split_x<<<grid_for(n * nrhs), 256, 0, s>>>(x, ldx, n, (int)nrhs, xhi, xlo, st);
    EBV_TRY(launch_ok());
    prof::Scope ps(s, prof::kResidual, 2.0 * n * (d->kl + d->ku + 1) * nrhs);
    k_band_residual_df<<<ceil_div(n, 8), 256, 0, s>>>(a_orig, d->ld, n, d->kl, d->ku, lower, xhi, xlo, (int)nrhs,
                                                       bs, nrhs, r, nrhs, rmax, st);
    return launch_ok();
  };
  if (d->storage == EBV_PROFILE || d->storage == EBV_DENSE_SYM) {
    const bool dsym = d->storage == EBV_DENSE_SYM;
    auto aview = [&](auto *p) {
      using E = std::remove_pointer_t<decltype(p)>;
      return dsym ? dense_symlo_view(p, d->ld) : profile_view<E>(p, n, d->kl, d->ku);
    };
    auto presidual = [&](const double *x, int64_t ldx, float *xhi, float *xlo, const double *bs, double *r,
                         unsigned long long *rmax, DevStatus *st, bool) -> ebv_status_t {
      k_split_x<<<grid_for(n * nrhs), 256, 0, s>>>(x, ldx, n, (int)nrhs, xhi, xlo, st);
      EBV_TRY(launch_ok());
      prof::Scope ps(s, prof::kResidual, 2.0 * n * (dsym ? n : d->kl + d->ku + 1) * nrhs);
      k_view_residual_df<<<ceil_div(n, 8), 256, 0, s>>>(aview(const_cast<double *>(a_orig)), n, xhi, xlo,
                                                         (int)nrhs, bs, nrhs, r, nrhs, rmax, st);
      return launch_ok();
    };
    if (fp64)
      return solve_refined<double>(aview((double *)lu), n, b, nrhs, ldb, refine, rep, (char *)ws, L, true, presidual,
                                   s);
    if (prec == EBV_FP32)
      return solve_refined<float>(aview((float *)lu), n, b, nrhs, ldb, refine, rep, (char *)ws, L, false, presidual,
                                  s);
    return EBV_ERR_UNSUPPORTED;
  }
  // b_double: FP64 right-hand sides and solution (FP64 factors, or the
  // mixed precisions' FP32 factors); FP32 ones for EBV_FP32
  auto run = [&](auto *p, bool b_double) {
    return lower ? solve_refined(symlo_view(p, d->ld, d->kl), n, b, nrhs, ldb, refine, rep, (char *)ws, L, b_double,
                                 residual, s)
                 : solve_refined(band_view(p, d->ld, d->kl, d->ku), n, b, nrhs, ldb, refine, rep, (char *)ws, L,
                                 b_double, residual, s);
  };
  if (fp64) return run((double *)lu, true);
  if (prec == EBV_FP32) return run((float *)lu, false);
  if (prec == EBV_MIXED_BF16 || prec == EBV_MIXED_FP16) return run((float *)lu, true);
  return EBV_ERR_UNSUPPORTED;
}

// Small dense FP64 systems: the panel loop above on a dense view (64-column
// panels: the diagonal block alone on one CTA, L21 / U12 by substitution on
// many, one trailing update), without the envelope scan.
ebv_status_t dense_small_factor(double *a, int64_t ld, int64_t n, int32_t *info, void *ws, cudaStream_t s) {
  return band_factor_t<double>(dense_view(a, ld), n, info, nullptr, nullptr, false, nullptr, s, false);
}

}  // namespace ebv

// ---------------------------------------------------------------------------
// Profile storage from a row band (host).
// ---------------------------------------------------------------------------
using namespace ebv;

extern "C" ebv_status_t ebv_profile_from_band(int64_t n, int64_t kl, int64_t ku, const double *ab, int64_t ldab,
                                              ebv_prec_t prec, void *out, size_t out_bytes, size_t *bytes_needed,
                                              int64_t *kl_out, int64_t *ku_out) {
  if (n < 1 || kl < 0 || ku < 0 || kl >= n || ku >= n || ldab < kl + ku + 1 || !ab) return EBV_ERR_ARG;
  if (prec != EBV_FP64 && prec != EBV_FP32) return EBV_ERR_UNSUPPORTED;
  const int64_t nb = (n + kNB - 1) / kNB;
  const size_t es = prec == EBV_FP64 ? 8 : 4;
  auto a = [&](int64_t i, int64_t j) { return ab[i * ldab + (j - i + kl)]; };
  // First non-zero left of the diagonal block over each row block, and
  // above it over each column block (the diagonal block is kept whole).
  std::vector<int32_t> lo((size_t)nb), up((size_t)nb);
  int64_t klp = 0, kup = 0;
  for (int64_t b = 0; b < nb; ++b) {
    const int64_t r0 = b * kNB, r1 = std::min<int64_t>(n, r0 + kNB);
    int64_t first = r0;
    for (int64_t i = r0; i < r1; ++i)
      for (int64_t j = std::max<int64_t>(0, i - kl); j < std::min<int64_t>(first, r0); ++j)
        if (a(i, j) != 0.0) {
          first = j;
          break;
        }
    lo[b] = (int32_t)first;
    int64_t top = r0;  // column block b: first row above the diagonal block with a non-zero
    for (int64_t j = r0; j < r1; ++j)
      for (int64_t i = std::max<int64_t>(0, j - ku); i < std::min<int64_t>(top, r0); ++i)
        if (a(i, j) != 0.0) {
          top = i;
          break;
        }
    up[b] = (int32_t)top;
    klp = std::max<int64_t>(klp, r1 - 1 - first);
    kup = std::max<int64_t>(kup, r1 - 1 - top);
  }
  klp = std::min<int64_t>(klp, n - 1);
  kup = std::min<int64_t>(kup, n - 1);
  std::vector<int64_t> offL((size_t)nb), offU((size_t)nb);
  int64_t count = 0;
  for (int64_t b = 0; b < nb; ++b) {
    offL[b] = count;
    count += (int64_t)kNB * ((b + 1) * kNB - lo[b]);
  }
  for (int64_t c = 0; c < nb; ++c) {
    offU[c] = count;
    count += (int64_t)kNB * (c * kNB - up[c]);
  }
  const size_t need = profile_header_bytes(n) + (size_t)count * es;
  if (bytes_needed) *bytes_needed = need;
  if (kl_out) *kl_out = klp;
  if (ku_out) *ku_out = kup;
  if (!out) return EBV_OK;
  if (out_bytes < need) return EBV_ERR_WORKSPACE;
  char *h = (char *)out;
  std::memset(h, 0, need);
  std::memcpy(h, lo.data(), 4 * (size_t)nb);
  std::memcpy(h + 4 * nb, up.data(), 4 * (size_t)nb);
  std::memcpy(h + 8 * nb, offL.data(), 8 * (size_t)nb);
  std::memcpy(h + 16 * nb, offU.data(), 8 * (size_t)nb);
  char *vals = h + profile_header_bytes(n);
  auto put = [&](int64_t off, double v) {
    if (es == 8)
      ((double *)vals)[off] = v;
    else
      ((float *)vals)[off] = (float)v;
  };
  for (int64_t b = 0; b < nb; ++b)  // lower parts with the diagonal blocks (rows past n stay 0)
    for (int64_t i = b * kNB; i < std::min<int64_t>(n, (b + 1) * kNB); ++i)
      for (int64_t j = lo[b]; j < std::min<int64_t>(n, (b + 1) * kNB); ++j)
        if (j - i >= -kl && j - i <= ku) put(offL[b] + (i - b * kNB) * ((b + 1) * kNB - lo[b]) + (j - lo[b]), a(i, j));
  for (int64_t c = 0; c < nb; ++c)  // parts above the diagonal blocks
    for (int64_t i = up[c]; i < c * kNB; ++i)
      for (int64_t j = c * kNB; j < std::min<int64_t>(n, (c + 1) * kNB); ++j)
        if (j - i <= ku) put(offU[c] + (i - up[c]) * kNB + (j - c * kNB), a(i, j));
  return EBV_OK;
}
