// Tensor-core (tcgen05) trailing update of the mixed-precision factorisation:
//
//   C(m0+i, n0+j) -= scale * sum_{k<K} lb(m0+i, k0+k) * ut(n0+j, k0+k)
//
// i.e. K aggregated rank-1 updates of Eq. 6c with bfloat16 / half operands
// and FP32 accumulation.  lb holds L (row-major) and ut holds U^T, so both
// operands are K-major.
//
// One 128 x BN output tile per CTA of 6 warps:
//   warp 0      TMA producer: 128x64 A and BNx64 B slabs, 128-byte swizzle,
//               into a STAGES-deep ring guarded by full/empty mbarriers;
//   warp 1      allocates BN TMEM columns; one lane issues tcgen05.mma
//               (M=128, N=BN, K=16) into the TMEM accumulator and commits
//               each slab back to its empty barrier;
//   warps 2..5  epilogue: tcgen05.ld of the accumulator (warp w reads TMEM
//               lanes 32*(w%4)...), C -= scale * D in FP32, with the loads of
//               C issued ahead (the first ones while the MMAs still run).
// Every mbarrier wait is bounded; on expiry the CTA records EBV_ERR_TIMEOUT,
// drains its own TMA copies and MMAs (bounded), frees TMEM and returns.
#include <cuda.h>

#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "tcgen05.cuh"

namespace ebv {

namespace {

constexpr int BM = 128, BK = 64, STAGES = 4, NTHREADS = 192;

// Instruction descriptor of kind::f16: FP32 accumulator, A and B of the same
// 16-bit type (fmt 0 = half, 1 = bfloat16), both K-major, M = 128, N = n.
constexpr uint32_t make_idesc(uint32_t fmt, int n) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

template <int BN>
constexpr int smem_bytes() {
  return STAGES * (BM * BK * 2 + BN * BK * 2) + 1024 /* alignment slack */ + 256 /* barriers */;
}

template <int BN>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_tc_update(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, float *C, int64_t ldc,
                const float *scale, int64_t m0, int64_t n0, int k0, int M, int N, int KB, uint32_t idesc, int vec_ok,
                DevStatus *st) {
  constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2, STAGE_BYTES = A_BYTES + B_BYTES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *full = (uint64_t *)(base + STAGES * STAGE_BYTES);
  uint64_t *empty = full + STAGES;
  uint64_t *tfull = empty + STAGES;
  uint32_t *tmem_holder = (uint32_t *)(tfull + 1);
  volatile int *abort_flag = (volatile int *)(tmem_holder + 1);
  auto stage_a = [&](int s) { return base + s * STAGE_BYTES; };
  auto stage_b = [&](int s) { return base + s * STAGE_BYTES + A_BYTES; };

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  // Grouped raster: consecutive CTAs sweep the N tiles of a group of GROUP_M
  // M tiles, so one wave touches ~GROUP_M A slabs and a few B slabs, which
  // stay in L2 instead of streaming all of B from HBM once per wave.
  constexpr int GROUP_M = 16;
  const int num_m = (M + BM - 1) / BM, num_n = (N + BN - 1) / BN;
  const int bid = blockIdx.x;
  const int group = bid / (GROUP_M * num_n);
  const int first_m = group * GROUP_M;
  const int gsize = min(GROUP_M, num_m - first_m);
  const int within = bid % (GROUP_M * num_n);
  const int tile_m = first_m + within % gsize, tile_n = within / gsize;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(tfull, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                 "r"(BN)
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

  if (warp == 0 && lane == 0) {
    // ---- TMA producer ----
    const int ya = (int)(m0 + (int64_t)tile_m * BM), yb = (int)(n0 + (int64_t)tile_n * BN);
    int issued = 0;
    for (int kb = 0; kb < KB; ++kb) {
      const int s = kb % STAGES, u = kb / STAGES;
      if (u > 0 && !mbar_wait(&empty[s], (u - 1) & 1, abort_flag)) {
        fail(1);
        break;
      }
      mbar_expect_tx(&full[s], STAGE_BYTES);
      tma_load_2d(stage_a(s), &tmA, &full[s], k0 + kb * BK, ya);
      tma_load_2d(stage_b(s), &tmB, &full[s], k0 + kb * BK, yb);
      issued = kb + 1;
    }
    // Our own copies must have landed before the CTA may exit.
    for (int kb = issued - STAGES > 0 ? issued - STAGES : 0; kb < issued; ++kb)
      if (!mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1, nullptr)) set_status(st, EBV_ERR_TIMEOUT, 2);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    for (int kb = 0; kb < KB; ++kb) {
      const int s = kb % STAGES, u = kb / STAGES;
      if (!mbar_wait(&full[s], u & 1, abort_flag)) {
        fail(3);
        break;
      }
      tc_fence_after();
      const uint64_t adesc = sw128_desc(smem_u32(stage_a(s)));
      const uint64_t bdesc = sw128_desc(smem_u32(stage_b(s)));
#pragma unroll
      for (int k = 0; k < BK / 16; ++k)  // +32 bytes along K inside the swizzle atom
        umma_f16(tmem, adesc + 2 * k, bdesc + 2 * k, idesc, (kb | k) != 0 ? 1u : 0u);
      umma_commit(&empty[s]);
    }
    umma_commit(tfull);
    if (!mbar_wait(tfull, 0, nullptr)) set_status(st, EBV_ERR_TIMEOUT, 4);  // MMAs retired before TMEM is freed
  } else if (warp >= 2) {
    // ---- epilogue ----
    // C does not depend on the accumulator: the first PF 16-column chunks of
    // this thread's row of C are loaded before the MMAs finish, and every
    // chunk's store is followed by the load of the chunk PF ahead, so PF
    // loads are always in flight instead of one round trip per chunk.
    constexpr int NCH = BN / 16, PF = NCH < 4 ? NCH : 4;
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const int64_t gi = m0 + (int64_t)tile_m * BM + row;
    const bool row_ok = gi < m0 + M;
    float *crow = C + gi * ldc;
    const int64_t jbase = n0 + (int64_t)tile_n * BN;
    auto fast = [&](int ci) { return row_ok && vec_ok && jbase + ci * 16 + 16 <= n0 + N; };
    float4 cb[PF][4];
    auto fetch = [&](int ci, float4 (&d)[4]) {
      if (fast(ci)) {
        const float4 *p = reinterpret_cast<const float4 *>(crow + jbase + ci * 16);
#pragma unroll
        for (int v = 0; v < 4; ++v) d[v] = p[v];
      }
    };
#pragma unroll
    for (int p = 0; p < PF; ++p) fetch(p, cb[p]);
    if (mbar_wait(tfull, 0, abort_flag)) {
      tc_fence_after();
      const float inv = scale[2];
#pragma unroll 1
      for (int c = 0; c < NCH; c += PF) {
#pragma unroll
        for (int p = 0; p < PF; ++p) {
          const int ci = c + p;
          uint32_t r[16];
          __syncwarp();  // tcgen05.ld is warp-collective: reconverge after the divergent stores
          tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ci * 16), r);
          const int64_t gj0 = jbase + ci * 16;
          if (fast(ci)) {
            float4 *dst = reinterpret_cast<float4 *>(crow + gj0);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
              float4 x = cb[p][v];
              x.x -= __uint_as_float(r[4 * v + 0]) * inv;
              x.y -= __uint_as_float(r[4 * v + 1]) * inv;
              x.z -= __uint_as_float(r[4 * v + 2]) * inv;
              x.w -= __uint_as_float(r[4 * v + 3]) * inv;
              dst[v] = x;
            }
          } else if (row_ok && gj0 < n0 + N) {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (gj0 + j < n0 + N) crow[gj0 + j] -= __uint_as_float(r[j]) * inv;
          }
          if (ci + PF < NCH) fetch(ci + PF, cb[p]);
        }
      }
    } else {
      fail(5);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
}

// ---------------------------------------------------------------------------
// The same update for small K (at most CS_MAXKB slabs), with the C tile in
// shared memory: with few slabs the update is bound by moving C (read and
// written once, FP32), and a per-thread register prefetch keeps too few
// bytes in flight to cover the memory latency.  Here the producer also
// TMA-loads the whole 128 x 128 FP32 tile of C (four 32-column blocks,
// 128-byte swizzle) while the MMAs run; the epilogue subtracts the
// accumulator in shared memory and TMA-stores the blocks back (the map's
// extent clips the ragged edges).  Four operand stages of 32 KB + 64 KB of C.
// ---------------------------------------------------------------------------
constexpr int CS_BN = 128, CS_STAGES = 4, CS_MAXKB = 8, CS_CB = 32;  // CS_CB: columns per C block (128 bytes)
constexpr int cs_smem_bytes() {
  return CS_STAGES * (BM * BK * 2 + CS_BN * BK * 2) + BM * CS_BN * 4 + 1024 /* alignment */ + 256 /* barriers */;
}

__global__ void __launch_bounds__(NTHREADS, 1)
    k_tc_update_cs(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmC, const float *scale, int64_t m0, int64_t n0, int k0, int M,
                   int N, int KB, uint32_t idesc, DevStatus *st) {
  constexpr int BN = CS_BN, A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2, STAGE_BYTES = A_BYTES + B_BYTES;
  constexpr int CBLK_BYTES = BM * CS_CB * 4, NCB = BN / CS_CB;  // 16 KB per 32-column block
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *cs = base + CS_STAGES * STAGE_BYTES;  // C tile: NCB blocks of 128 rows x 128 bytes
  uint64_t *full = (uint64_t *)(cs + BM * BN * 4);
  uint64_t *empty = full + CS_STAGES;
  uint64_t *tfull = empty + CS_STAGES;
  uint64_t *cfull = tfull + 1;
  uint32_t *tmem_holder = (uint32_t *)(cfull + 1);
  volatile int *abort_flag = (volatile int *)(tmem_holder + 1);
  auto stage_a = [&](int s) { return base + s * STAGE_BYTES; };
  auto stage_b = [&](int s) { return base + s * STAGE_BYTES + A_BYTES; };

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int num_n = (N + BN - 1) / BN;
  const int tile_m = blockIdx.x / num_n, tile_n = blockIdx.x % num_n;
  const int ya = (int)(m0 + (int64_t)tile_m * BM), xb = (int)(n0 + (int64_t)tile_n * BN);

  if (threadIdx.x == 0) {
    for (int s = 0; s < CS_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(tfull, 1);
    mbar_init(cfull, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                 "r"(BN)
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

  if (warp == 0 && lane == 0) {
    // ---- TMA producer: every operand slab (KB <= CS_STAGES * 2), then C ----
    int issued = 0;
    bool c_issued = false;
    for (int kb = 0; kb < KB; ++kb) {
      const int s = kb % CS_STAGES, u = kb / CS_STAGES;
      if (u > 0 && !mbar_wait(&empty[s], (u - 1) & 1, abort_flag)) {
        fail(21);
        break;
      }
      mbar_expect_tx(&full[s], STAGE_BYTES);
      tma_load_2d(stage_a(s), &tmA, &full[s], k0 + kb * BK, ya);
      tma_load_2d(stage_b(s), &tmB, &full[s], k0 + kb * BK, xb);
      issued = kb + 1;
      if (kb == CS_STAGES - 1 || kb == KB - 1) {  // the first ring of slabs is in flight: C next
        if (!c_issued) {
          mbar_expect_tx(cfull, BM * BN * 4);
          for (int j = 0; j < NCB; ++j) tma_load_2d(cs + j * CBLK_BYTES, &tmC, cfull, xb + j * CS_CB, ya);
          c_issued = true;
        }
      }
    }
    // Our own copies must have landed before the CTA may exit.
    for (int kb = issued - CS_STAGES > 0 ? issued - CS_STAGES : 0; kb < issued; ++kb)
      if (!mbar_wait(&full[kb % CS_STAGES], (kb / CS_STAGES) & 1, nullptr)) set_status(st, EBV_ERR_TIMEOUT, 22);
    if (c_issued && !mbar_wait(cfull, 0, nullptr)) set_status(st, EBV_ERR_TIMEOUT, 23);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    for (int kb = 0; kb < KB; ++kb) {
      const int s = kb % CS_STAGES, u = kb / CS_STAGES;
      if (!mbar_wait(&full[s], u & 1, abort_flag)) {
        fail(24);
        break;
      }
      tc_fence_after();
      const uint64_t adesc = sw128_desc(smem_u32(stage_a(s)));
      const uint64_t bdesc = sw128_desc(smem_u32(stage_b(s)));
#pragma unroll
      for (int k = 0; k < BK / 16; ++k)
        umma_f16(tmem, adesc + 2 * k, bdesc + 2 * k, idesc, (kb | k) != 0 ? 1u : 0u);
      umma_commit(&empty[s]);
    }
    umma_commit(tfull);
    if (!mbar_wait(tfull, 0, nullptr)) set_status(st, EBV_ERR_TIMEOUT, 25);
  } else if (warp >= 2) {
    // ---- epilogue: C -= inv * D in shared memory, then TMA stores ----
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const bool ok = mbar_wait(tfull, 0, abort_flag) && mbar_wait(cfull, 0, abort_flag);
    if (__all_sync(0xffffffffu, ok)) {
      tc_fence_after();
      const float inv = scale[2];
#pragma unroll 1
      for (int h = 0; h < BN / 16; ++h) {
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * 16), r);
        uint8_t *blk = cs + (h / 2) * CBLK_BYTES + row * 128;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c16 = (h % 2) * 4 + u;  // 16-byte chunk of the 128-byte row
          float4 *p = reinterpret_cast<float4 *>(blk + ((c16 ^ (row & 7)) << 4));
          float4 x = *p;
          x.x -= __uint_as_float(r[4 * u + 0]) * inv;
          x.y -= __uint_as_float(r[4 * u + 1]) * inv;
          x.z -= __uint_as_float(r[4 * u + 2]) * inv;
          x.w -= __uint_as_float(r[4 * u + 3]) * inv;
          *p = x;
        }
      }
      fence_proxy_async_smem();  // the tile's generic-proxy writes, before the async-proxy stores
    } else {
      fail(26);
    }
    asm volatile("bar.sync 1, 128;" ::: "memory");  // the four epilogue warps
    if (warp == 2 && lane == 0 && !*abort_flag) {
      for (int j = 0; j < NCB; ++j) tma_store_2d(&tmC, cs + j * CBLK_BYTES, xb + j * CS_CB, ya);
      bulk_commit();
      bulk_wait_all();  // the stores are done before the CTA exits
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

bool make_map(CUtensorMap *map, int op, const void *base, int64_t cols, int64_t rows, int64_t ld_elems, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld_elems * 2};
  const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(map, op == 0 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                        const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// FP32 map of C (extent: columns < n0 + N, rows < m0 + M, so TMA stores stop
// at the update's edges), 32 x 128 boxes with the 128-byte swizzle.
bool make_map_c(CUtensorMap *map, const float *C, int64_t ldc, int64_t cols, int64_t rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ldc * 4};
  const cuuint32_t box[2] = {(cuuint32_t)CS_CB, (cuuint32_t)BM};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(C), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

ebv_status_t launch_tc_cs(int op, float *C, int64_t ldc, const void *lb, const void *ut, int64_t ldsh,
                          const float *scale, int64_t m0, int64_t n0, int64_t k0, int64_t M, int64_t N, int64_t K,
                          DevStatus *st, cudaStream_t s) {
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] { attr_err = set_smem(k_tc_update_cs, cs_smem_bytes()); });
  if (attr_err != cudaSuccess) return EBV_ERR_CUDA;
  CUtensorMap ma, mb, mc;
  if (!make_map(&ma, op, lb, k0 + K, m0 + M, ldsh, BM)) return EBV_ERR_UNSUPPORTED;
  if (!make_map(&mb, op, ut, k0 + K, n0 + N, ldsh, CS_BN)) return EBV_ERR_UNSUPPORTED;
  if (!make_map_c(&mc, C, ldc, n0 + N, m0 + M)) return EBV_ERR_UNSUPPORTED;
  const dim3 grid(ceil_div(N, CS_BN) * ceil_div(M, BM));
  k_tc_update_cs<<<grid, NTHREADS, cs_smem_bytes(), s>>>(ma, mb, mc, scale, m0, n0, (int)k0, (int)M, (int)N,
                                                         (int)(K / BK), make_idesc(op == 0 ? 1u : 0u, CS_BN), st);
  return launch_ok();
}

template <int BN>
ebv_status_t launch_tc(int op, float *C, int64_t ldc, const void *lb, const void *ut, int64_t ldsh, const float *scale,
                       int64_t m0, int64_t n0, int64_t k0, int64_t M, int64_t N, int64_t K, DevStatus *st,
                       cudaStream_t s) {
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    attr_err = set_smem(k_tc_update<BN>, smem_bytes<BN>());
  });
  if (attr_err != cudaSuccess) return EBV_ERR_CUDA;
  CUtensorMap ma, mb;
  if (!make_map(&ma, op, lb, k0 + K, m0 + M, ldsh, BM)) return EBV_ERR_UNSUPPORTED;
  if (!make_map(&mb, op, ut, k0 + K, n0 + N, ldsh, BN)) return EBV_ERR_UNSUPPORTED;
  const int vec_ok = (ldc % 4 == 0) && (n0 % 4 == 0) && (((uintptr_t)C) % 16 == 0);
  dim3 grid(ceil_div(N, BN) * ceil_div(M, BM));  // linear; the kernel maps it with a grouped raster
  k_tc_update<BN><<<grid, NTHREADS, smem_bytes<BN>(), s>>>(ma, mb, C, ldc, scale, m0, n0, (int)k0, (int)M, (int)N,
                                                          (int)(K / BK), make_idesc(op == 0 ? 1u : 0u, BN), vec_ok, st);
  return launch_ok();
}

}  // namespace

bool tc_available() { return encode_fn() != nullptr; }

bool make_map_bf16(CUtensorMap *map, const void *base, int64_t cols, int64_t rows, int64_t ld_elems, int box_cols,
                   int box_rows, int swizzle_bytes) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld_elems * 2};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUtensorMapSwizzle sw = swizzle_bytes == 128  ? CU_TENSOR_MAP_SWIZZLE_128B
                                : swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                : swizzle_bytes == 32 ? CU_TENSOR_MAP_SWIZZLE_32B
                                                      : CU_TENSOR_MAP_SWIZZLE_NONE;
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

ebv_status_t tc_update(int op, float *C, int64_t ldc, const void *lb, const void *ut, int64_t ldsh,
                       const float *scale, int64_t m0, int64_t n0, int64_t k0, int64_t M, int64_t N, int64_t K,
                       DevStatus *st, cudaStream_t s) {
  // Shapes the kernel takes: whole 64-wide K slabs, 16-byte aligned rows and
  // slab origins (TMA), coordinates inside int range.
  if (K <= 0 || K % BK != 0 || k0 % 8 != 0 || (ldsh * 2) % 16 != 0) return EBV_ERR_UNSUPPORTED;
  if (((uintptr_t)lb) % 16 != 0 || ((uintptr_t)ut) % 16 != 0) return EBV_ERR_UNSUPPORTED;
  if (m0 + M > INT32_MAX || n0 + N > INT32_MAX || k0 + K > INT32_MAX) return EBV_ERR_UNSUPPORTED;
  // Few K slabs: C staged in shared memory by TMA (16-byte aligned rows and origin).
  if (K / BK <= CS_MAXKB && N > 64 && ldc % 4 == 0 && n0 % 4 == 0 && ((uintptr_t)C) % 16 == 0)
    return launch_tc_cs(op, C, ldc, lb, ut, ldsh, scale, m0, n0, k0, M, N, K, st, s);
  if (N >= 192) return launch_tc<256>(op, C, ldc, lb, ut, ldsh, scale, m0, n0, k0, M, N, K, st, s);
  if (N > 64) return launch_tc<128>(op, C, ldc, lb, ut, ldsh, scale, m0, n0, k0, M, N, K, st, s);
  return launch_tc<64>(op, C, ldc, lb, ut, ldsh, scale, m0, n0, k0, M, N, K, st, s);
}

}  // namespace ebv
