// Shared helpers for the EbV CUDA library (sm_103a).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstddef>

#include "ebv.h"
#include "profile.h"

namespace ebv {

// Leaf block size of the dense and banded factorisations (columns handled by
// one diagonal-block kernel).
constexpr int kNB = 64;

// Bound on the polls of any device-side wait (each poll sleeps ~100 ns), so a
// wait that never completes ends in well under a second with EBV_ERR_TIMEOUT.
constexpr long long kSpinLimit = 1LL << 22;

// Device status block kept at the start of every workspace.
struct DevStatus {
  int32_t code;   // ebv_status_t of the first device-side failure (0 = none)
  int32_t where;  // kernel-specific detail (e.g. the block that timed out)
  int32_t done;   // refinement: set once the stop test has passed
  int32_t pad;
  int32_t arrive;  // arrival counter of last-CTA hand-offs; back at 0 when each such launch ends
  int32_t pad2;
};
constexpr size_t kStatusBytes = 256;  // keeps what follows 256-byte aligned

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

#define EBV_TRY(expr)                       \
  do {                                      \
    ebv_status_t s_ = (expr);               \
    if (s_ != EBV_OK) return s_;            \
  } while (0)

#define EBV_CU(expr)                        \
  do {                                      \
    cudaError_t e_ = (expr);                \
    if (e_ != cudaSuccess) return EBV_ERR_CUDA; \
  } while (0)

inline ebv_status_t launch_ok() {
  prof::count_launch();
  return cudaGetLastError() == cudaSuccess ? EBV_OK : EBV_ERR_CUDA;
}

// Opt a kernel into `bytes` of dynamic shared memory (if > 0) with the
// maximum shared-memory carveout.  Every kernel of the library asks for the
// same carveout, so consecutive launches never make the SMs reconfigure their
// L1 / shared-memory split between kernels.
template <typename K>
inline cudaError_t set_smem(K kernel, int bytes) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       (int)cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess && bytes > 0) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}

__host__ __device__ inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }
__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

// ---------------------------------------------------------------------------
// Conversions between the working types and the tensor-core operand types.
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T from_float(float x);
template <> __device__ __forceinline__ float from_float<float>(float x) { return x; }
template <> __device__ __forceinline__ __nv_bfloat16 from_float<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <> __device__ __forceinline__ __half from_float<__half>(float x) { return __float2half_rn(x); }

__device__ __forceinline__ float to_float(float x) { return x; }
__device__ __forceinline__ float to_float(double x) { return (float)x; }
__device__ __forceinline__ float to_float(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ float to_float(__half x) { return __half2float(x); }

// Reciprocal of a pivot.  It is always formed in FP64 (the pivots'
// reciprocals are among the few FP64 operations of the mixed-precision
// paths); the binary32 factorisations round it once to binary32 and scale
// their L vectors with it (Eq. 6a).  Measured on GB300: a dependent FP64
// reciprocal of one warp takes about as long as the IEEE binary32 one (~88
// cycles per pivot step), so the FP64 form costs nothing extra on the chain.
__device__ __forceinline__ double pivot_rcp(double p) { return 1.0 / p; }
__device__ __forceinline__ float pivot_rcp(float p) { return (float)(1.0 / (double)p); }
// A zero or non-finite pivot (tested in the working precision), on the bit
// pattern: zero of either sign, or the all-ones exponent of Inf / NaN (no
// floating-point compare on the pivot chain).
__device__ __forceinline__ bool pivot_bad(double p) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(p);
  return (b << 1) == 0ull || ((b >> 52) & 0x7FFull) == 0x7FFull;
}
__device__ __forceinline__ bool pivot_bad(float p) {
  const unsigned int b = __float_as_uint(p);
  return (b << 1) == 0u || ((b >> 23) & 0xFFu) == 0xFFu;
}

// Record the first device-side failure in a status block (first writer wins).
__device__ __forceinline__ void set_status(DevStatus *st, int code, int where) {
  if (st && atomicCAS(&st->code, 0, code) == 0) st->where = where;
}

// Acquire load of a flag written by another CTA.
__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bounded wait until *flag >= want (acquire).  Gives up after `polls` polls,
// or early once the status block reports a failure elsewhere; on expiry it
// records EBV_ERR_TIMEOUT with `where` and returns false.  Every inter-CTA
// wait of the library goes through here.
__device__ __forceinline__ bool bounded_wait_geq(const int *flag, int want, DevStatus *st, long long polls,
                                                 int where) {
  for (long long it = 0; it < polls; ++it) {
    if (ld_acquire(flag) >= want) return true;
    if ((it & 255) == 255 && st && ld_acquire(&st->code) != 0) return false;
    if (it >= 32) __nanosleep(64);  // a short hot spin first: the flag is usually close
  }
  set_status(st, EBV_ERR_TIMEOUT, where);
  return false;
}

}  // namespace ebv
