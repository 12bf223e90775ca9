// Dense factorisation and solve: host-side orchestration of the kernels.
//
// Factorisation: recursive column-halving Doolittle (no pivoting).  A panel of
// w columns is factored by factoring its left half, computing the U vectors of
// the left half's rows for the right half (U12 = L11^{-1} A12), applying the
// aggregated rank-1 updates of Eq. 6c to the right half (A22 -= L21 U12, one
// GEMM with K = w/2) and factoring the right half.  The leaves are 64-column
// blocks: an equal bi-vectorised diagonal-block kernel (Eq. 6-7) plus the
// row-parallel L21 = A21 U11^{-1}.  Compared with a fixed-width right-looking
// loop, the halving keeps most flops in GEMMs with a large K, which moves the
// FP32 working matrix through HBM O(log n) times instead of O(n / nb) times.
#include <algorithm>

#include "internal.h"
#include "solve_driver.cuh"

namespace ebv {

namespace {

// ---------------------------------------------------------------------------
// Conversion of A to the FP32 working matrix and the power-of-two operand
// scales of the half-precision tensor-core path.
// ---------------------------------------------------------------------------
// FP32 working copy of columns [c0, c1) of A (n x n, row-major, leading
// dimension n for the copy), with the largest off-diagonal and smallest
// diagonal magnitude folded into maxoff / mindiag.  Rows are strided over the
// grid, columns over the threads (no index division).
__global__ void k_to_working(const double *a, int64_t lda, int64_t n, int64_t c0, int64_t c1, float *w,
                             unsigned int *maxoff, unsigned int *mindiag) {
  unsigned int lmax = 0u, lmin = 0x7F800000u;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    const double *src = a + i * lda;
    float *dst = w + i * n;
    for (int64_t j = c0 + threadIdx.x; j < c1; j += blockDim.x) {
      const float v = (float)src[j];
      dst[j] = v;
      const unsigned int bits = __float_as_uint(fabsf(v));
      if (i == j)
        lmin = min(lmin, bits);
      else
        lmax = max(lmax, bits);
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, off));
    lmin = min(lmin, __shfl_xor_sync(0xffffffffu, lmin, off));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(maxoff, lmax);
    atomicMin(mindiag, lmin);
  }
}

// Converts the columns of A into the FP32 working copy in order, as the
// factorisation first needs them.  With `ev` set, block b of cbw columns is
// converted only after ev[b] (its host-to-device copy) has completed, so the
// copy of the right part of A overlaps the factorisation of the left part.
struct ColumnStager {
  const double *a;
  int64_t lda, n;
  float *w;
  unsigned int *scan;
  cudaStream_t s;
  const cudaEvent_t *ev;  // null: A is already on the device
  int64_t cbw;
  bool convert = true;    // false: the copies also wrote the working copy and the scan
  int64_t done = 0;
  ebv_status_t ensure(int64_t c_hi) {
    c_hi = std::min<int64_t>(c_hi, n);
    while (done < c_hi) {
      const int64_t c1 = std::min<int64_t>(n, done + cbw);
      if (ev) EBV_CU(cudaStreamWaitEvent(s, ev[done / cbw], 0));
      if (convert) {
        k_to_working<<<(int)std::min<int64_t>(n, 4096), 256, 0, s>>>(a, lda, n, done, c1, w, scan, scan + 1);
        EBV_TRY(launch_ok());
      }
      done = c1;
    }
    return EBV_OK;
  }
};

// scale = [sL, sU, 1/(sL sU), -].  bfloat16 shares FP32's exponent range and
// needs no scaling.  For half, L and U entries are bounded here by the largest
// off-diagonal |a_ij| (over the smallest |a_ii| for L); each is scaled by the
// power of two that brings that bound to 2^10, well inside half's normal range
// [6.1e-5, 65504].  Powers of two make the scaling and the unscaling exact.
__global__ void k_make_scale(int op, const unsigned int *maxoff, const unsigned int *mindiag, float *scale) {
  float sl = 1.f, su = 1.f;
  if (op == 1) {
    const float mo = __uint_as_float(*maxoff);
    float md = __uint_as_float(*mindiag);
    if (!(md > 0.f) || isinf(md)) md = 1.f;
    if (mo > 0.f && isfinite(mo)) {
      int el = (int)floorf(log2f(1024.f * md / mo));
      int eu = (int)floorf(log2f(1024.f / mo));
      el = max(-40, min(40, el));
      eu = max(-40, min(40, eu));
      sl = ldexpf(1.f, el);
      su = ldexpf(1.f, eu);
    }
  }
  scale[0] = sl;
  scale[1] = su;
  scale[2] = (float)(1.0 / ((double)sl * (double)su));
  scale[3] = 0.f;
}

template <typename T>
struct SimtGemm;
template <>
struct SimtGemm<double> {
  static constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
};
template <>
struct SimtGemm<float> {
  static constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8;
};

}  // namespace

// ---------------------------------------------------------------------------
// Mixed-precision GEMM dispatch.
// ---------------------------------------------------------------------------
static int g_lowp_mode = 0;
// Small dense FP64 factorisations as substitution panels (true) or on one
// thread-block cluster (false); testing hook ebv_debug_set_small_dense.
static bool g_small_dense_panels = true;
void set_small_dense_panels(bool on) { g_small_dense_panels = on; }
void set_lowp_gemm_mode(int mode) { g_lowp_mode = mode; }
int get_lowp_gemm_mode() { return g_lowp_mode; }

ebv_status_t simt_update(int op, float *C, int64_t ldc, const void *lb, const void *ut, int64_t ldsh,
                         const float *scale, int64_t m0, int64_t n0, int64_t k0, int64_t M, int64_t N, int64_t K,
                         cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0) return EBV_OK;
  constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8;
  dim3 grid(ceil_div(N, BN), ceil_div(M, BM));
  if (op == 0)
    k_gemm_nt_simt<__nv_bfloat16, BM, BN, BK, TM, TN><<<grid, 256, 0, s>>>(
        C, ldc, (const __nv_bfloat16 *)lb, (const __nv_bfloat16 *)ut, ldsh, scale, m0, n0, k0, M, N, K);
  else
    k_gemm_nt_simt<__half, BM, BN, BK, TM, TN><<<grid, 256, 0, s>>>(C, ldc, (const __half *)lb, (const __half *)ut,
                                                                    ldsh, scale, m0, n0, k0, M, N, K);
  return launch_ok();
}

ebv_status_t lowp_update(int op, float *C, int64_t ldc, const void *lb, const void *ut, int64_t ldsh,
                         const float *scale, int64_t m0, int64_t n0, int64_t k0, int64_t M, int64_t N, int64_t K,
                         DevStatus *dst, cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0) return EBV_OK;
  prof::Scope ps(s, prof::kLowpGemm, 2.0 * M * N * K);
  if (g_lowp_mode != 1) {
    ebv_status_t st = tc_update(op, C, ldc, lb, ut, ldsh, scale, m0, n0, k0, M, N, K, dst, s);
    if (st != EBV_ERR_UNSUPPORTED) return st;
  }
  return simt_update(op, C, ldc, lb, ut, ldsh, scale, m0, n0, k0, M, N, K, s);
}

// ---------------------------------------------------------------------------
// Recursive factorisation.
// ---------------------------------------------------------------------------
namespace {

template <typename T, typename SH>
struct Factorizer {
  MatView<T> A;
  int64_t n;
  int32_t *info;
  cudaStream_t s;
  Shadow<SH> sh;
  int op;  // -1: working-precision SIMT updates; 0/1: bf16/half tensor-core updates
  DevStatus *st = nullptr;
  T *inv = nullptr;  // per leaf: L11^{-1} then U11^{-1} (2 * 64 * 64 entries)
  ColumnStager *stg = nullptr;  // mixed precisions: makes columns available on first use
  int *flags = nullptr;         // binary32: one zeroed flag per leaf for the fused diagonal-block launches

  ebv_status_t need(int64_t c_hi) { return stg ? stg->ensure(c_hi) : EBV_OK; }

  // CTAs of a fused launch that can be co-resident (0 if unknown).
  template <typename K>
  static int coop_capacity(K kernel, size_t smem) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, 256, smem) != cudaSuccess) {
      (void)cudaGetLastError();
      return 0;
    }
    return sms * per;
  }
  template <typename K, typename... Args>
  ebv_status_t launch_coop(K kernel, int grid, size_t smem, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    EBV_CU(cudaLaunchKernelEx(&cfg, kernel, args...));
    return launch_ok();
  }
  // Grid of a fused launch over `rows` rows below a leaf, if it fits co-resident (else 0).
  int fused_grid(bool update, int64_t rows) const {
    if constexpr (sizeof(T) != 4) {
      return 0;
    } else {
      if (!flags || rows <= 0) return 0;
      constexpr size_t smem = diag_fused_smem_bytes<T, kNB>();
      static const int cap_l21 = coop_capacity(k_diag_l21<T, SH, kNB>, smem);
      static const int cap_upd = coop_capacity(k_diag_l21_update<T, SH, kNB>, smem);
      const int64_t grid = 1 + (rows + kNB - 1) / kNB;
      return grid <= (update ? cap_upd : cap_l21) ? (int)grid : 0;
    }
  }
  // Whether a k_diag_l21_u12 grid fits co-resident.
  bool u12_fits(int64_t grid) const {
    if constexpr (sizeof(T) != 4) {
      return false;
    } else {
      static const int cap = coop_capacity(k_diag_l21_u12<T, SH, kNB>, diag_fused_smem_bytes<T, kNB>());
      return flags && grid <= cap;
    }
  }

  static int64_t split(int64_t w) {  // leaf-aligned first half of a w-wide range
    const int64_t nb = (w + kNB - 1) / kNB;
    return ((nb + 1) / 2) * kNB;
  }
  T *leaf_inv(int64_t c0) const { return inv + (c0 / kNB) * 2 * kNB * kNB; }

  // The diagonal block of the leaf at c0, then (with_l21) its L21 for every row below.
  ebv_status_t leaf(int64_t c0, int w, bool with_l21 = true) {
    constexpr size_t smem = pair_smem_bytes<T, kNB>();
    EBV_TRY(need(c0 + w));
    if (with_l21) {
      if (const int grid = fused_grid(false, n - c0 - w)) {  // one cooperative launch
        prof::Scope ps(s, prof::kPanel, 2.0 * w * w * w / 3.0 + 2.0 * (n - c0 - w) * w * w);
        return launch_coop(k_diag_l21<T, SH, kNB>, grid, diag_fused_smem_bytes<T, kNB>(), A, c0, w, n, info,
                           leaf_inv(c0), sh, flags + c0 / kNB, st);
      }
    }
    {
      prof::Scope ps(s, prof::kPanel, 2.0 * w * w * w / 3.0);
      k_diag_factor<T, kNB, 4 * kNB><<<1, 4 * kNB, diagb_smem_bytes<T, kNB>(), s>>>(A, c0, w, info, leaf_inv(c0));
      EBV_TRY(launch_ok());
    }
    const int64_t rb = c0 + w, re = n;
    if (with_l21 && re > rb) {
      prof::Scope ps(s, prof::kL21, 2.0 * (re - rb) * w * w);
      if (sizeof(T) == 8 && ceil_div(re - rb, kNB) < 152)  // FP64, fewer 64-row tiles than SMs: 16-row strips
        k_trsm_ru_strip<T, SH, kNB, 16><<<ceil_div(re - rb, 16), 256, smem, s>>>(A, c0, w, rb, re, leaf_inv(c0), sh);
      else
        k_trsm_ru<T, SH, kNB><<<ceil_div(re - rb, kNB), 256, smem, s>>>(A, c0, w, rb, re, leaf_inv(c0), sh);
      EBV_TRY(launch_ok());
    }
    return EBV_OK;
  }

  ebv_status_t gemm(int64_t m0, int64_t n0, int64_t k0, int64_t M, int64_t N, int64_t K) {
    if (M <= 0 || N <= 0 || K <= 0) return EBV_OK;
    EBV_TRY(need(n0 + N));
    if (op >= 0)
      return lowp_update(op, (float *)A.base, A.ld, sh.lb, sh.ut, sh.ld, sh.scale, m0, n0, k0, M, N, K, st, s);
    using G = SimtGemm<T>;
    prof::Scope ps(s, prof::kSimtGemm, 2.0 * M * N * K);
    dim3 grid(ceil_div(N, G::BN), ceil_div(M, G::BM));
    k_gemm_nn<T, G::BM, G::BN, G::BK, G::TM, G::TN>
        <<<grid, (G::BM / G::TM) * (G::BN / G::TN), 0, s>>>(A, m0, n0, k0, M, N, K);
    return launch_ok();
  }

  // U(r0 .. r0+h, cl .. ch) = L(r0.., r0..)^{-1} A(r0.., cl..ch)
  ebv_status_t trsm_ll(int64_t r0, int64_t h, int64_t cl, int64_t ch) {
    if (ch <= cl || h <= 0) return EBV_OK;
    EBV_TRY(need(ch));
    if (h <= kNB) {
      prof::Scope ps(s, prof::kTrsm, 2.0 * h * h * (ch - cl));
      k_trsm_ll<T, SH, kNB><<<ceil_div(ch - cl, kNB), 256, pair_smem_bytes<T, kNB>(), s>>>(A, r0, (int)h, cl, ch,
                                                                                         leaf_inv(r0), sh);
      return launch_ok();
    }
    if (h <= kTrsmMaxBlocks * kNB) {
      // Narrower column strips when there are few columns: more CTAs, each
      // with a shorter chain of tile products.
      prof::Scope ps(s, prof::kTrsm, 1.0 * h * h * (ch - cl));
      constexpr size_t smem = trsm_multi_smem_bytes<T, kNB, kTrsmMaxBlocks>();
      const int64_t N = ch - cl;
      if (N >= 64 * 148) {
        k_trsm_ll_multi<T, SH, kNB, kTrsmMaxBlocks, 64><<<ceil_div(N, 64), 256, smem, s>>>(A, r0, (int)h, cl, ch, leaf_inv(r0), sh);
      } else if (sizeof(T) == 4 && A.ld % 4 == 0 && ((uintptr_t)A.base) % 16 == 0) {
        // binary32 with 16-byte rows: everything resident in shared memory
        if constexpr (sizeof(T) == 4) {
          // At most one wave: a CTA keeps its copy of L11's tiles for every
          // strip it takes (the copy is most of a strip's time).
          constexpr size_t rsm = trsm_res_smem_bytes<kNB, kTrsmMaxBlocks>();
          static const int wave = coop_capacity(k_trsm_ll_resident<SH, kNB, kTrsmMaxBlocks>, rsm);
          const int strips = ceil_div(N, kResCW);
          k_trsm_ll_resident<SH, kNB, kTrsmMaxBlocks><<<wave > 0 ? std::min(strips, wave) : strips, 256, rsm, s>>>(
              A, r0, (int)h, cl, ch, leaf_inv(r0), sh);
        }
      } else if (N >= 32 * 148) {
        k_trsm_ll_multi<T, SH, kNB, kTrsmMaxBlocks, 32><<<ceil_div(N, 32), 256, smem, s>>>(A, r0, (int)h, cl, ch, leaf_inv(r0), sh);
      } else {
        k_trsm_ll_multi<T, SH, kNB, kTrsmMaxBlocks, 16><<<ceil_div(N, 16), 256, smem, s>>>(A, r0, (int)h, cl, ch, leaf_inv(r0), sh);
      }
      return launch_ok();
    }
    const int64_t h1 = split(h);
    EBV_TRY(trsm_ll(r0, h1, cl, ch));
    EBV_TRY(gemm(r0 + h1, cl, r0, h - h1, ch - cl, h1));
    return trsm_ll(r0 + h1, h - h1, cl, ch);
  }

  // Factor columns c0 .. c0+w of rows c0 .. n.
  ebv_status_t rlu(int64_t c0, int64_t w) {
    if (w <= kNB) return leaf(c0, (int)w);
    const int64_t w1 = split(w);
    if (w <= 2 * kNB) {  // two leaves: U12 and the trailing update in one launch
      // binary32: the left leaf's L21 joins that launch as well
      constexpr bool fuse_l21 = sizeof(T) == 4;
      const int64_t rows = n - c0 - w1;
      if (const int grid = fused_grid(true, rows)) {  // and the left leaf's diagonal block too
        EBV_TRY(need(c0 + w));
        prof::Scope ps(s, prof::kPanel,
                       2.0 * w1 * w1 * w1 / 3.0 + 2.0 * rows * w1 * w1 + 2.0 * w1 * w1 * (w - w1) +
                           2.0 * rows * w1 * (w - w1));
        EBV_TRY(launch_coop(k_diag_l21_update<T, SH, kNB>, grid, diag_fused_smem_bytes<T, kNB>(), A, c0, (int)w1,
                            (int)(w - w1), n, info, leaf_inv(c0), sh, flags + c0 / kNB, st));
        return leaf(c0 + w1, (int)(w - w1));
      }
      EBV_TRY(leaf(c0, (int)w1, !fuse_l21));
      EBV_TRY(need(c0 + w));
      if (fuse_l21) {
        prof::Scope ps(s, prof::kLeafUpdate,
                       2.0 * rows * w1 * w1 + 2.0 * w1 * w1 * (w - w1) + 2.0 * rows * w1 * (w - w1));
        k_leaf_ru_update<T, SH, kNB><<<ceil_div(rows, kNB), 256, leaf_ru_update_smem_bytes<T, kNB>(), s>>>(
            A, c0, (int)w1, (int)(w - w1), n, leaf_inv(c0), sh, st);
        EBV_TRY(launch_ok());
      } else {
        prof::Scope ps(s, prof::kLeafUpdate, 2.0 * w1 * w1 * (w - w1) + 2.0 * rows * w1 * (w - w1));
        k_leaf_update<T, SH, kNB><<<ceil_div(rows, kNB), 256, leaf_update_smem_bytes<T, kNB>(), s>>>(
            A, c0, (int)w1, (int)(w - w1), n, leaf_inv(c0), sh, st);
        EBV_TRY(launch_ok());
      }
      return leaf(c0 + w1, (int)(w - w1));
    }
    if (w1 == 2 * kNB && w <= 4 * kNB) {
      // The left half is two full leaves: the first as one fused launch, the
      // second fused with this node's U12 (columns c0+w1 .. c0+w).
      const int64_t rows1 = n - c0 - kNB, rows2 = n - c0 - w1;
      const int g1 = fused_grid(true, rows1);
      const int nl = ceil_div(rows2, kNB), nu = ceil_div(w - w1, 16);
      if (g1 && u12_fits(1 + nl + nu)) {
        EBV_TRY(need(c0 + w));
        {
          prof::Scope ps(s, prof::kPanel,
                         2.0 * kNB * kNB * kNB / 3.0 + 2.0 * rows1 * kNB * kNB * 2.0 + 2.0 * rows1 * kNB * kNB);
          EBV_TRY(launch_coop(k_diag_l21_update<T, SH, kNB>, g1, diag_fused_smem_bytes<T, kNB>(), A, c0, (int)kNB,
                              (int)kNB, n, info, leaf_inv(c0), sh, flags + c0 / kNB, st));
        }
        {
          prof::Scope ps(s, prof::kPanel,
                         2.0 * kNB * kNB * kNB / 3.0 + 2.0 * rows2 * kNB * kNB + 1.0 * w1 * w1 * (w - w1));
          EBV_TRY(launch_coop(k_diag_l21_u12<T, SH, kNB>, 1 + nl + nu, diag_fused_smem_bytes<T, kNB>(), A, c0,
                              (int)kNB, n, nl, c0 + w1, c0 + w, info, (const T *)leaf_inv(c0), leaf_inv(c0 + kNB),
                              sh, flags + (c0 + kNB) / kNB, st));
        }
        EBV_TRY(gemm(c0 + w1, c0 + w1, c0, n - c0 - w1, w - w1, w1));
        return rlu(c0 + w1, w - w1);
      }
    }
    EBV_TRY(rlu(c0, w1));
    EBV_TRY(trsm_ll(c0, w1, c0 + w1, c0 + w));
    EBV_TRY(gemm(c0 + w1, c0 + w1, c0, n - c0 - w1, w - w1, w1));
    return rlu(c0 + w1, w - w1);
  }
};

struct DenseFactorLayout {
  size_t inv, flags, lb, ut, scale, scan, total;
  int64_t ldsh;  // shadow row stride: a multiple of 64 elements (128 B), as TMA wants 16-byte strides
};

DenseFactorLayout factor_layout(int64_t n, ebv_prec_t prec) {
  DenseFactorLayout L{};
  size_t off = kStatusBytes;
  L.ldsh = (n + 63) / 64 * 64;
  const size_t leaves = (size_t)((n + kNB - 1) / kNB);
  L.inv = off;
  off = align256(off + leaves * 2 * kNB * kNB * (prec == EBV_FP64 ? 8 : 4));
  L.flags = off;
  off = align256(off + leaves * sizeof(int));
  if (prec == EBV_MIXED_BF16 || prec == EBV_MIXED_FP16) {
    L.lb = off; off = align256(off + (size_t)n * L.ldsh * 2);
    L.ut = off; off = align256(off + (size_t)n * L.ldsh * 2);
    L.scale = off; off = align256(off + 16);
    L.scan = off; off = align256(off + 16);
  }
  L.total = off;
  return L;
}

}  // namespace

size_t dense_factor_ws(int64_t n, ebv_prec_t prec) { return factor_layout(n, prec).total; }
size_t dense_solve_ws(int64_t n, int64_t nrhs, ebv_prec_t prec) {
  return solve_layout(n, nrhs, prec == EBV_FP64 ? 8 : 4, true).total;
}

// Mixed-precision factorisation of A (FP64, device, leading dimension lda)
// into the FP32 working copy / factors `lowp` (leading dimension n).  ev /
// cbw: see ColumnStager (null: all of A is already on the device).
static ebv_status_t dense_factor_mixed(int64_t n, ebv_prec_t prec, const double *a, int64_t lda, float *lowp,
                                      int32_t *info, char *w, const DenseFactorLayout &L, const cudaEvent_t *ev,
                                      int64_t cbw, bool convert, cudaStream_t s) {
  DevStatus *dst = (DevStatus *)w;
  unsigned int *scan = (unsigned int *)(w + L.scan);
  float *scale = (float *)(w + L.scale);
  if (convert) {
    EBV_CU(cudaMemsetAsync(scan, 0, 4, s));         // max |a_ij|, i != j: starts at +0
    EBV_CU(cudaMemsetAsync(scan + 1, 0x7F, 4, s));  // min |a_ii|: starts at 0x7F7F7F7F (3.4e38)
  }
  static const bool carveout = (set_smem(k_to_working, 0), set_smem(k_make_scale, 0), true);
  (void)carveout;
  ColumnStager stg{a, lda, n, lowp, scan, s, ev, ev ? cbw : n, convert};
  const int op = prec == EBV_MIXED_BF16 ? 0 : 1;
  // bfloat16 needs no operand scaling; half's scale comes from all of A.
  if (op == 1) EBV_TRY(stg.ensure(n));
  k_make_scale<<<1, 1, 0, s>>>(op, scan, scan + 1, scale);
  EBV_TRY(launch_ok());
  float *inv = (float *)(w + L.inv);
  int *flags = (int *)(w + L.flags);
  EBV_CU(cudaMemsetAsync(flags, 0, sizeof(int) * (size_t)((n + kNB - 1) / kNB), s));
  if (op == 0) {
    EBV_TRY((prepare_leaf_kernels<float, __nv_bfloat16>()));
    Factorizer<float, __nv_bfloat16> f{
        dense_view(lowp, n), n, info, s,
        Shadow<__nv_bfloat16>{(__nv_bfloat16 *)(w + L.lb), (__nv_bfloat16 *)(w + L.ut), L.ldsh, scale}, 0, dst, inv,
        &stg, flags};
    EBV_TRY(f.rlu(0, n));
    return stg.ensure(n);
  }
  EBV_TRY((prepare_leaf_kernels<float, __half>()));
  Factorizer<float, __half> f{dense_view(lowp, n), n, info, s,
                              Shadow<__half>{(__half *)(w + L.lb), (__half *)(w + L.ut), L.ldsh, scale}, 1, dst, inv,
                              &stg, flags};
  return f.rlu(0, n);
}

ebv_status_t dense_factor(const ebv_desc_t *d, ebv_prec_t prec, void *a, void *lowp, int32_t *info, void *ws,
                          size_t ws_bytes, cudaStream_t s) {
  const int64_t n = d->n;
  EBV_CU(cudaMemsetAsync(info, 0, sizeof(int32_t), s));
  if (ws) EBV_CU(cudaMemsetAsync(ws, 0, sizeof(DevStatus), s));
  if (n == 0) return EBV_OK;
  const DenseFactorLayout L = factor_layout(n, prec);
  if (!ws || ws_bytes < L.total) return EBV_ERR_WORKSPACE;
  char *w = (char *)ws;
  DevStatus *dst = (DevStatus *)ws;
  const Shadow<float> none{nullptr, nullptr, 0, nullptr};
  if (prec == EBV_FP64 && n <= kSmallDenseMaxN && g_small_dense_panels) {
    // Small FP64 systems as 64-column panels: the diagonal block factored
    // alone, L21 / U12 by substitution (no FP64 inverses on the chain).
    return dense_small_factor((double *)a, d->ld, n, info, ws, s);
  }
  if ((prec == EBV_FP64 || prec == EBV_FP32) && n <= kClusterDenseMaxN) {
    // A small system whole on one thread-block cluster (one launch).
    const ebv_status_t st =
        cluster_panel(prec == EBV_FP64, a, d->ld, kDenseBand, kDenseBand, false, 0, (int)n, n, 0, info, nullptr, s);
    if (st != EBV_ERR_UNSUPPORTED) return st;
  }
  if (prec == EBV_FP64) {
    EBV_TRY((prepare_leaf_kernels<double, float>()));
    Factorizer<double, float> f{dense_view((double *)a, d->ld), n, info, s, none, -1, dst, (double *)(w + L.inv)};
    return f.rlu(0, n);
  }
  if (prec == EBV_FP32) {
    EBV_TRY((prepare_leaf_kernels<float, float>()));
    int *flags = (int *)(w + L.flags);
    EBV_CU(cudaMemsetAsync(flags, 0, sizeof(int) * (size_t)((n + kNB - 1) / kNB), s));
    Factorizer<float, float> f{dense_view((float *)a, d->ld), n,    info, s, none, -1, dst, (float *)(w + L.inv),
                               nullptr,                           flags};
    return f.rlu(0, n);
  }
  return dense_factor_mixed(n, prec, (const double *)a, d->ld, (float *)lowp, info, w, L, nullptr, 0, true, s);
}

// Scan words (largest off-diagonal, smallest diagonal magnitude) of the mixed
// factorisation inside its workspace, initialised on s, for copies that
// fill the working copy themselves (see ebv_gesv_host).
unsigned int *dense_factor_scan_init(int64_t n, ebv_prec_t prec, void *ws, cudaStream_t s) {
  unsigned int *scan = (unsigned int *)((char *)ws + factor_layout(n, prec).scan);
  if (cudaMemsetAsync(scan, 0, 4, s) != cudaSuccess || cudaMemsetAsync(scan + 1, 0x7F, 4, s) != cudaSuccess)
    return nullptr;
  return scan;
}

// Mixed-precision factorisation whose A is still arriving: block b of cbw
// columns is on the device once ev[b] has completed (see ebv_gesv_host).
// convert: the factorisation converts each block to FP32 itself; otherwise
// the copies already wrote the working copy and the scan words.
ebv_status_t dense_factor_staged(int64_t n, ebv_prec_t prec, const double *a_dev, float *lowp, int32_t *info,
                                 void *ws, size_t ws_bytes, const cudaEvent_t *ev, int64_t cbw, bool convert,
                                 cudaStream_t s) {
  EBV_CU(cudaMemsetAsync(info, 0, sizeof(int32_t), s));
  if (ws) EBV_CU(cudaMemsetAsync(ws, 0, sizeof(DevStatus), s));
  if (n == 0) return EBV_OK;
  const DenseFactorLayout L = factor_layout(n, prec);
  if (!ws || ws_bytes < L.total) return EBV_ERR_WORKSPACE;
  if (prec != EBV_MIXED_BF16 && prec != EBV_MIXED_FP16) return EBV_ERR_UNSUPPORTED;
  return dense_factor_mixed(n, prec, a_dev, n, lowp, info, (char *)ws, L, ev, cbw, convert, s);
}

// R = B - A X for the dense refinement: on the tensor cores (exact digit
// splitting) where TMA is available, else the triple-binary32 SIMT kernel.
static ebv_status_t dense_residual(const double *a, int64_t lda, int64_t n, const double *x, int64_t ldx, int64_t nrhs,
                            const double *b, double *r, unsigned long long *rmax, char *w, const DenseSolveLayout &L,
                            bool first, DevStatus *st, cudaStream_t s) {
  if (tc_available())
    return residual_tc(a, lda, n, x, ldx, nrhs, b, nrhs, r, nrhs, rmax, w + L.tcres, !first, st, s);
  float *xhi = (float *)(w + L.xhi), *xlo = (float *)(w + L.xlo);
  k_split_x<<<grid_for(n * nrhs), 256, 0, s>>>(x, ldx, n, (int)nrhs, xhi, xlo, st);
  EBV_TRY(launch_ok());
  constexpr int RB = 32, RC = 32, KC = 32;
  dim3 grid(ceil_div(n, RB), ceil_div(nrhs, RC));
  prof::Scope ps(s, prof::kResidual, 2.0 * n * n * nrhs);
  k_residual_df<RB, RC, KC><<<grid, 256, 0, s>>>(a, lda, n, xhi, xlo, (int)nrhs, b, nrhs, r, nrhs, rmax, st);
  return launch_ok();
}

// R = B - A X with the refinement's residual kernel (testing hook).
ebv_status_t debug_residual(int64_t n, const double *a, int64_t lda, const double *x, const double *b, int64_t nrhs,
                            double *r, void *ws, size_t ws_bytes, cudaStream_t s) {
  const DenseSolveLayout L = solve_layout(n, nrhs, 8, true);
  if (!ws || ws_bytes < L.total) return EBV_ERR_WORKSPACE;
  char *w = (char *)ws;
  DevStatus *st = (DevStatus *)w;
  EBV_CU(cudaMemsetAsync(ws, 0, sizeof(DevStatus), s));
  unsigned long long *rmax = (unsigned long long *)(w + L.rmax);
  EBV_CU(cudaMemsetAsync(rmax, 0, nrhs * 8, s));
  return dense_residual(a, lda, n, x, nrhs, nrhs, b, r, rmax, w, L, true, st, s);
}

ebv_status_t dense_solve(const ebv_desc_t *d, ebv_prec_t prec, const void *lu, const double *a_orig, void *b,
                         int64_t nrhs, int64_t ldb, const ebv_refine_t *refine, ebv_refine_report_t *rep, void *ws,
                         size_t ws_bytes, cudaStream_t s) {
  const int64_t n = d->n;
  const bool fp64 = prec == EBV_FP64;
  const DenseSolveLayout L = solve_layout(n, nrhs, fp64 ? 8 : 4, true);
  if (!ws || ws_bytes < L.total) return EBV_ERR_WORKSPACE;
  EBV_CU(cudaMemsetAsync(ws, 0, sizeof(DevStatus), s));
  if (n == 0 || nrhs == 0) return EBV_OK;
  char *w = (char *)ws;
  auto residual = [&](const double *x, int64_t ldx, float *, float *, const double *bs, double *r,
                      unsigned long long *rmax, DevStatus *st, bool first) -> ebv_status_t {
    return dense_residual(a_orig, d->ld, n, x, ldx, nrhs, bs, r, rmax, w, L, first, st, s);
  };
  const bool b_double = prec != EBV_FP32;
  if (fp64 && !refine && n <= kSmallSolveMaxN && nrhs <= 8 && g_small_dense_panels) {
    // small systems: direct block substitution in one CTA (no diagonal-block inverses)
    prof::Scope ps(s, prof::kTrsv, 2.0 * n * n * nrhs);
    k_small_solve<double><<<1, 256, 0, s>>>(dense_view((double *)lu, d->ld), (int)n, (double *)b, ldb, (int)nrhs);
    return launch_ok();
  }
  if (fp64)
    return solve_refined<double>(dense_view((double *)lu, d->ld), n, b, nrhs, ldb, refine, rep, w, L, b_double,
                                 residual, s);
  const int64_t ldf = (prec == EBV_FP32) ? d->ld : n;
  return solve_refined<float>(dense_view((float *)lu, ldf), n, b, nrhs, ldb, refine, rep, w, L, b_double, residual, s);
}

}  // namespace ebv
