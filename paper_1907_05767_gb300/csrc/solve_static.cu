// ebv_solve_static: ebv_solve for callers that may not allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs while a stream is being
// captured into a CUDA graph by someone else, real-time loops whose memory is
// budgeted up front, plug-ins whose host application owns every allocation,
// or a caller that has no allocator handle of its own.  For them the solve's
// workspace lives in a file-scope device array of fixed size, which the CUDA
// module reserves when this library is loaded on a device and keeps until the
// process exits.  The caller still passes the factors, the right-hand sides
// and (optionally) the refinement inputs and report.
//
// The array is shared by every call on a device and keeps the previous
// call's contents.  The solve path clears what must start at zero (status
// word, substitution flags, the refinement's column maxima) on every call.
// Two calls whose work overlaps on the GPU (different streams, or different
// host threads without ordering) race on the array.
#include <mutex>

#include "internal.h"

namespace ebv {
namespace {

// Bytes of the static workspace; with n <= EBV_STATIC_MAX_N and
// nrhs <= EBV_STATIC_MAX_NRHS every precision and storage fits (FP64 with
// refinement at the limits needs about 16.5 MiB).
constexpr size_t kStaticBytes = EBV_STATIC_SCRATCH_BYTES;

// Device-side workspace.  In host code this name is only a stand-in for the
// symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_ws[kStaticBytes];

constexpr int kMaxDevices = 64;

// The array's address belongs to the CUDA context that loaded this library's
// module on the device: after cudaDeviceReset the primary context, and the
// module in it, are made anew, and a caller may make a context of its own
// current on the same device.  So the address is cached per device together
// with the CUDA driver's unique ID of the context it was looked up in, and looked
// up again whenever the current context's ID differs.
struct Slot {
  unsigned long long ctx_id = 0;  // 0: nothing cached
  void *ptr = nullptr;
};
Slot g_slot[kMaxDevices];
std::mutex g_mutex;

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// Unique ID of the current context (0 if there is none or it cannot be read).
unsigned long long current_ctx_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (CtxGetCurrentFn)p;
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (CtxGetIdFn)p;
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// Device address of g_static_ws in the current context of the current
// device.  The first call in a context looks it up (cudaGetSymbolAddress,
// which also makes the device's primary context current if none is); later
// calls in the same context reuse it.
ebv_status_t static_ws(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return EBV_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return EBV_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mutex);
  Slot &slot = g_slot[dev];
  unsigned long long id = current_ctx_id();
  if (id == 0 || id != slot.ctx_id) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_ws) != cudaSuccess || !p) return EBV_ERR_CUDA;
    id = current_ctx_id();  // the lookup may have made the primary context current
    if (id == 0) return EBV_ERR_CUDA;
    slot.ctx_id = id;
    slot.ptr = p;
  }
  *out = slot.ptr;
  return EBV_OK;
}

}  // namespace
}  // namespace ebv

using namespace ebv;

extern "C" ebv_status_t ebv_solve_static(const ebv_desc_t *desc, ebv_prec_t prec, const void *lu,
                                         const double *a_orig, void *b, int64_t nrhs, int64_t ldb,
                                         const ebv_refine_t *refine, ebv_refine_report_t *report_dev,
                                         ebv_stream_t stream) {
  if (!desc) return EBV_ERR_ARG;
  // Sizes beyond the static array are rejected before any device work.
  if (desc->n > EBV_STATIC_MAX_N || nrhs > EBV_STATIC_MAX_NRHS) return EBV_ERR_WORKSPACE;
  if (desc->n < 0 || nrhs < 0) return EBV_ERR_ARG;
  const size_t need = desc->storage != EBV_DENSE ? band_solve_ws(desc->n, nrhs, prec)
                                                : dense_solve_ws(desc->n, nrhs, prec);
  if (need > kStaticBytes) return EBV_ERR_WORKSPACE;
  void *ws = nullptr;
  const ebv_status_t st = static_ws(&ws);
  if (st != EBV_OK) return st;
  return ebv_solve(desc, prec, lu, a_orig, b, nrhs, ldb, refine, report_dev, ws, kStaticBytes, stream);
}
