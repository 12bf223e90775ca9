// Panel factorisation on a thread-block cluster (Eq. 6a-c on one panel, with
// the column pairing of Eq. 7 across the cluster's CTAs).
//
// A panel is the W columns [c0, c0+W) of rows [c0, c0+R) (R >= W), plus the
// U12 block: the same first W rows in the U columns right of the panel.  The
// kernel runs the W elimination steps of the panel unblocked: step k divides
// the L vector of column k by the pivot (Eq. 6a) and subtracts the rank-1
// product from every later panel column (all R rows) and from the U12 columns
// (the panel's own rows only, which is U12 = L11^{-1} A12).  The result is the
// packed L\U of the W x W diagonal block, L21 for rows W..R-1 and U12, so the
// caller only has the trailing update left.
//
// Ownership: the panel's columns go to the NC CTAs of one cluster as the
// pairs {p, W-1-p} (pair p to CTA p mod NC), a long column with a short one,
// so every CTA does about the same work over the W steps (Eq. 7); U12 is cut
// into NC contiguous column chunks (every U12 column costs the same).  Each
// CTA holds its columns in shared memory, column-major.  Per step, the CTAs
// copy pivot column k from its owner through distributed shared memory
// (ld.shared::cluster via cooperative_groups), scale the pivot row of their
// own columns by 1/a_kk (formed in FP64, once, by the owner during the
// previous step) and update.  The owner scales column k into L one step
// later, after every CTA has copied it.  One cluster barrier per step orders
// all of this; there is no spin-wait anywhere (hardware barriers only).
//
// Used for band panels (R = W + kl rows, U = ku columns) and for a whole
// small dense matrix (W = R = n, U = 0).
#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace ebv {
namespace {

constexpr int kPT = 256;  // threads per CTA
// Panels taller than this read the pivot column from L2 (bcast) when the
// caller passes the scratch.
constexpr int kBcastMinRows = 256;

struct PanelShape {
  int nc;      // CTAs in the cluster
  int W;       // panel columns
  int R;       // panel rows (>= W)
  int U;       // U12 columns
  int slots;   // panel-column slots per CTA: 2 * ceil(ceil(W/2) / nc)
  int uc;      // U12 columns per CTA: ceil(U / nc)
};

__host__ __device__ inline PanelShape panel_shape(int nc, int W, int R, int U) {
  const int pairs = (W + 1) / 2;
  return PanelShape{nc, W, R, U, 2 * ((pairs + nc - 1) / nc), (U + nc - 1) / nc};
}

// Shared memory of one CTA, in elements of T: the panel columns (slots x R),
// the U12 columns (uc x W), pivot column k (R), the scaled pivot row of the
// own columns (slots + uc) and the pivot reciprocals of two consecutive steps.
template <typename T>
__host__ __device__ inline size_t panel_smem_elems(const PanelShape &p) {
  return (size_t)p.slots * p.R + (size_t)p.uc * p.W + p.R + p.slots + p.uc + 2;
}

// Panel column j -> (owner CTA, local slot).
__device__ __forceinline__ void col_home(int j, int W, int nc, int &owner, int &slot) {
  const int p = min(j, W - 1 - j);
  owner = p % nc;
  slot = 2 * (p / nc) + (j == p ? 0 : 1);
}
// Local slot -> panel column (-1 if the slot is empty).
__device__ __forceinline__ int slot_col(int s, int rank, int W, int nc) {
  const int p = rank + nc * (s / 2);
  if (p >= (W + 1) / 2) return -1;
  if (s % 2 == 0) return p;
  return (W - 1 - p == p) ? -1 : W - 1 - p;
}

// Element (i, j) of the band view (base + i*ld + j, zero outside -kl..ku).
// symlo: only the lower half of a symmetric band is stored; the panel reads
// a_ij above the diagonal as a_ji and writes back the lower half (L and the
// pivots) only.
template <typename T>
struct BandRef {
  T *base;
  int64_t ld, kl, ku;
  bool symlo;
  __device__ __forceinline__ bool in(int64_t i, int64_t j) const { return j - i >= -kl && j - i <= ku; }
  __device__ __forceinline__ T load(int64_t i, int64_t j) const {
    if (!in(i, j)) return T(0);
    return (symlo && j > i) ? base[j * ld + i] : base[i * ld + j];
  }
  __device__ __forceinline__ bool writable(int64_t i, int64_t j) const { return in(i, j) && !(symlo && j > i); }
};

// SMAX: an upper bound on the panel-column slots of one CTA (ps.slots), so the
// scaled pivot row of the own columns lives in registers and a thread's row
// update is one batch of independent loads, fused multiply-adds and stores.
//
// bcast (global, 2 (R + 1) elements, or null): with tall panels the 16 CTAs'
// reads of pivot column k from its owner's shared memory are limited by that
// one SM's shared-memory bandwidth (1.6 us per step measured at R = 576 on
// GB300).  With bcast the owner also stores the finished column and its
// reciprocal to slot k & 1 of bcast (L2) and the others read it from there.
template <typename T, int SMAX>
__global__ void __launch_bounds__(kPT) k_cluster_panel(BandRef<T> A, int64_t c0, PanelShape ps, int32_t *info,
                                                       T *bcast) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int nc = ps.nc, W = ps.W, R = ps.R, U = ps.U, S = ps.slots, UC = ps.uc;
  extern __shared__ __align__(16) unsigned char smraw[];
  T *Pc = reinterpret_cast<T *>(smraw);  // [S][R]
  T *Uc = Pc + (size_t)S * R;            // [UC][W]
  T *Lk = Uc + (size_t)UC * W;           // pivot column k, rows 0..R-1
  T *Up = Lk + R;                        // scaled pivot row of the own columns: [S] then [UC]
  T *Rc = Up + S + UC;                   // Rc[k & 1]: reciprocal of pivot k (written by its owner)
  const int u0 = rank * UC, un = max(0, min(UC, U - u0));  // own U12 columns u0 .. u0+un-1

  // Load the own columns (element (c0+i, c0+j)); out-of-band entries read as 0.
  for (int e = threadIdx.x; e < S * R; e += kPT) {
    const int s = e / R, i = e % R;
    const int j = slot_col(s, rank, W, nc);
    Pc[e] = j >= 0 ? A.load(c0 + i, c0 + j) : T(0);
  }
  for (int e = threadIdx.x; e < un * W; e += kPT) {  // row-wise: consecutive threads, consecutive columns
    const int i = e / un, jj = e % un;
    Uc[jj * W + i] = A.load(c0 + i, c0 + W + u0 + jj);
  }
  __syncthreads();
  {  // reciprocal of the first pivot, by its owner (and column 0 to bcast)
    int o0, s0;
    col_home(0, W, nc, o0, s0);
    if (rank == o0) {
      if (threadIdx.x == 0) {
        const T p = Pc[(size_t)s0 * R + 0];
        Rc[0] = pivot_rcp(p);
        if (bcast) __stcg(bcast + R, Rc[0]);
        if (pivot_bad(p) && info) atomicCAS(info, 0, (int)(c0 + 1));
      }
      if (bcast)
        for (int i = 1 + threadIdx.x; i < R; i += kPT) __stcg(bcast + i, Pc[(size_t)s0 * R + i]);
    }
  }
  T r_prev = T(0);
  int prev_slot = -1;
  for (int k = 0; k < W; ++k) {
    cluster.sync();  // column k and its reciprocal are final; everyone is done with column k-1
    int ok, sk;
    col_home(k, W, nc, ok, sk);
    // Pivot k's reciprocal sits in slot k & 1 of its owner (Rc, and bcast):
    // the owner of column k+1 (the same CTA for the middle pair) writes slot
    // (k+1) & 1 during this step, and slot k & 1 again only after the next
    // barrier, when every CTA has read it.
    T rk;
    if (bcast) {  // from L2, past L1 (the slot was read two steps ago)
      const T *src = bcast + (size_t)(k & 1) * (R + 1);
      for (int i = k + 1 + threadIdx.x; i < R; i += kPT) Lk[i] = __ldcg(src + i);
      rk = __ldcg(src + R);
    } else {  // from the owner's shared memory
      const T *remote = cluster.map_shared_rank(Pc + (size_t)sk * R, ok);
      const T *rrem = cluster.map_shared_rank(Rc + (k & 1), ok);
      for (int i = k + 1 + threadIdx.x; i < R; i += kPT) Lk[i] = remote[i];
      rk = *rrem;
    }
    // The previous pivot column, now copied by every CTA, becomes L (Eq. 6a).
    if (prev_slot >= 0)
      for (int i = k + threadIdx.x; i < R; i += kPT) Pc[(size_t)prev_slot * R + i] *= r_prev;
    // Row k of the own columns right of the pivot, times 1/a_kk.
    for (int t = threadIdx.x; t < S + un; t += kPT) {
      if (t < S) {
        const int j = slot_col(t, rank, W, nc);
        Up[t] = (j > k) ? Pc[(size_t)t * R + k] * rk : T(0);
      } else {
        Up[S + (t - S)] = Uc[(size_t)(t - S) * W + k] * rk;
      }
    }
    __syncthreads();
    // The owner of column k+1 forms the next pivot's reciprocal first (thread
    // 0, which also updates row k+1 below, with the same fused multiply-add),
    // so the FP64 division overlaps the other warps' updates.
    if (k + 1 < W) {
      int on, sn;
      col_home(k + 1, W, nc, on, sn);
      if (rank == on && threadIdx.x == 0) {
        const T u = Up[sn], a = Pc[(size_t)sn * R + k + 1];
        const T p = u != T(0) ? fma(-Lk[k + 1], u, a) : a;  // exactly what the update below stores
        Rc[(k + 1) & 1] = pivot_rcp(p);
        if (bcast) __stcg(bcast + (size_t)((k + 1) & 1) * (R + 1) + R, Rc[(k + 1) & 1]);
        if (pivot_bad(p) && info) atomicCAS(info, 0, (int)(c0 + k + 2));
      }
    }
    // Eq. 6c: a_ij -= a_ik * (a_kj / a_kk), panel columns on rows k+1..R-1
    // (a thread per row, all of the CTA's columns at once) ...
    T u[SMAX];
#pragma unroll
    for (int q = 0; q < SMAX; ++q) u[q] = q < S ? Up[q] : T(0);
    for (int i = k + 1 + threadIdx.x; i < R; i += kPT) {
      const T l = Lk[i];
      T v[SMAX];
#pragma unroll
      for (int q = 0; q < SMAX; ++q) v[q] = (q < S && u[q] != T(0)) ? Pc[(size_t)q * R + i] : T(0);
#pragma unroll
      for (int q = 0; q < SMAX; ++q)
        if (q < S && u[q] != T(0)) Pc[(size_t)q * R + i] = fma(-l, u[q], v[q]);
    }
    // The owner of column k+1 puts that column, as each thread has just
    // updated its rows (the same rows as in the loop above), into the next
    // bcast slot; the readers take the rows below the next pivot.
    if (bcast && k + 1 < W) {
      int on, sn;
      col_home(k + 1, W, nc, on, sn);
      if (rank == on) {
        T *dst = bcast + (size_t)((k + 1) & 1) * (R + 1);
        for (int i = k + 1 + threadIdx.x; i < R; i += kPT) __stcg(dst + i, Pc[(size_t)sn * R + i]);
      }
    }
    // ... and U12 columns on the panel's rows k+1..W-1: thread (row ti,
    // column group tg) takes columns tg, tg+4, ... (a warp reads 32
    // consecutive rows of one column: no bank conflicts).
    {
      const int ti = threadIdx.x % 64, tg = threadIdx.x / 64;
      const int i = k + 1 + ti;
      if (i < W) {
        const T l = Lk[i];
        for (int jb = tg; jb < un; jb += 16) {
          T uu[4], vv[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int jj = jb + 4 * q;
            uu[q] = jj < un ? Up[S + jj] : T(0);
            vv[q] = jj < un ? Uc[(size_t)jj * W + i] : T(0);
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int jj = jb + 4 * q;
            if (jj < un) Uc[(size_t)jj * W + i] = fma(-l, uu[q], vv[q]);
          }
        }
      }
    }
    if (rank == ok) {
      prev_slot = sk;
      r_prev = rk;
    } else {
      prev_slot = -1;
    }
  }
  cluster.sync();  // no CTA reads another's shared memory after this
  if (prev_slot >= 0)
    for (int i = W + threadIdx.x; i < R; i += kPT) Pc[(size_t)prev_slot * R + i] *= r_prev;
  __syncthreads();
  for (int e = threadIdx.x; e < S * R; e += kPT) {
    const int s = e / R, i = e % R;
    const int j = slot_col(s, rank, W, nc);
    if (j >= 0 && A.writable(c0 + i, c0 + j)) A.base[(c0 + i) * A.ld + c0 + j] = Pc[e];
  }
  for (int e = threadIdx.x; e < un * W; e += kPT) {
    const int i = e / un, jj = e % un;
    const int64_t j = c0 + W + u0 + jj;
    if (A.writable(c0 + i, j)) A.base[(c0 + i) * A.ld + j] = Uc[jj * W + i];
  }
}

// Largest cluster (16, else 8) that the device can run with this shared
// memory, or 0.
// The kernel instance for a slot count: SMAX = 4, 8, 16 or 32 (null above).
template <typename T>
using PanelKernel = void (*)(BandRef<T>, int64_t, PanelShape, int32_t *, T *);
template <typename T>
PanelKernel<T> panel_kernel(int slots) {
  if (slots <= 4) return k_cluster_panel<T, 4>;
  if (slots <= 8) return k_cluster_panel<T, 8>;
  if (slots <= 16) return k_cluster_panel<T, 16>;
  if (slots <= 32) return k_cluster_panel<T, 32>;
  return nullptr;
}

template <typename T>
bool prepare_panel_kernels() {
  static std::once_flag once;
  static bool ok = false;
  std::call_once(once, [] {
    ok = true;
    for (int sl : {4, 8, 16, 32}) {
      auto kern = panel_kernel<T>(sl);
      ok = ok && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
           cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) == cudaSuccess &&
           cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared) == cudaSuccess;
    }
    (void)cudaGetLastError();
  });
  return ok;
}

// Largest cluster (16, else 8) that the device can run with the shared
// memory of that shape, or 0.
template <typename T>
int cluster_size_for(int W, int R, int U) {
  if (!prepare_panel_kernels<T>()) return 0;
  for (int nc : {16, 8}) {
    const PanelShape ps = panel_shape(nc, W, R, U);
    const size_t smem = panel_smem_elems<T>(ps) * sizeof(T);
    auto kern = panel_kernel<T>(ps.slots);
    if (smem > 227 * 1024 || !kern) continue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nc);
    cfg.blockDim = dim3(kPT);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)nc;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) == cudaSuccess && clusters > 0) return nc;
    (void)cudaGetLastError();
  }
  return 0;
}

template <typename T>
ebv_status_t cluster_panel_t(T *base, int64_t ld, int64_t kl, int64_t ku, bool symlo, int64_t c0, int W, int R, int U,
                             int32_t *info, T *bcast, cudaStream_t s) {
  const int nc = cluster_size_for<T>(W, R, U);
  if (nc == 0) return EBV_ERR_UNSUPPORTED;
  const PanelShape ps = panel_shape(nc, W, R, U);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nc);
  cfg.blockDim = dim3(kPT);
  cfg.dynamicSmemBytes = panel_smem_elems<T>(ps) * sizeof(T);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)nc;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  prof::Scope sc(s, prof::kPanel, 2.0 * (double)W * W * W / 3.0 + 2.0 * (double)(R - W) * W * W / 2.0 +
                                      (double)W * W * U);
  EBV_CU(cudaLaunchKernelEx(&cfg, panel_kernel<T>(ps.slots), BandRef<T>{base, ld, kl, ku, symlo}, c0, ps, info,
                            R > kBcastMinRows ? bcast : nullptr));
  return launch_ok();
}

}  // namespace

static bool g_cluster_panel = true;
void set_cluster_panel(bool on) { g_cluster_panel = on; }
bool cluster_panel_enabled() { return g_cluster_panel; }

bool cluster_panel_fits(bool fp64, int W, int64_t R, int64_t U) {
  if (W < 1 || W > 256 || R < W || R > (1 << 20) || U < 0 || U > (1 << 20)) return false;
  const size_t es = fp64 ? 8 : 4;
  return panel_smem_elems<double>(panel_shape(16, W, (int)R, (int)U)) * es <= 227 * 1024;
}

ebv_status_t cluster_panel(bool fp64, void *base, int64_t ld, int64_t kl, int64_t ku, bool symlo, int64_t c0, int W,
                           int64_t R, int64_t U, int32_t *info, void *bcast, cudaStream_t s) {
  if (!g_cluster_panel || !cluster_panel_fits(fp64, W, R, U) || (symlo && U != 0)) return EBV_ERR_UNSUPPORTED;
  if (fp64)
    return cluster_panel_t<double>((double *)base, ld, kl, ku, symlo, c0, W, (int)R, (int)U, info, (double *)bcast, s);
  return cluster_panel_t<float>((float *)base, ld, kl, ku, symlo, c0, W, (int)R, (int)U, info, (float *)bcast, s);
}

}  // namespace ebv
