// ebv_gesv_host: A X = B for A and B in host memory, with the host-to-device
// copy of A overlapped with the factorisation.  A is copied column block by
// column block on a second stream; the factorisation converts each block into
// its FP32 working copy only once that block's copy has completed (the
// recursion reaches the columns of A from left to right), so most of the
// transfer hides behind the factorisation of the columns already there.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace ebv {
namespace {

constexpr int kMaxCopyBlocks = 64;
constexpr int kMaxDevices = 64;

// Copy stream and events of one device, created on the first call there.
struct HostPipe {
  cudaStream_t cs = nullptr;
  cudaEvent_t fork = nullptr;
  cudaEvent_t ev[kMaxCopyBlocks + 1] = {};  // ev[b]: column block b of A copied; ev[kMaxCopyBlocks]: B copied
  bool ready = false;
};
HostPipe g_pipe[kMaxDevices];
std::mutex g_pipe_mutex;

ebv_status_t host_pipe(HostPipe **out) {
  int dev = 0;
  EBV_CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return EBV_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_pipe_mutex);
  HostPipe &p = g_pipe[dev];
  if (!p.ready) {
    EBV_CU(cudaStreamCreateWithFlags(&p.cs, cudaStreamNonBlocking));
    EBV_CU(cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming));
    for (cudaEvent_t &e : p.ev) EBV_CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    p.ready = true;
  }
  *out = &p;
  return EBV_OK;
}

struct HostLayout {
  size_t a, lowp, x, info, rep, ws, ws_bytes, total;
};
HostLayout host_layout(int64_t n, int64_t nrhs, ebv_prec_t prec) {
  HostLayout L{};
  size_t off = 0;
  L.a = off; off = align256(off + (size_t)n * n * 8);
  L.lowp = off; off = align256(off + (size_t)n * n * 4);
  L.x = off; off = align256(off + (size_t)n * std::max<int64_t>(nrhs, 1) * 8);
  L.info = off; off = align256(off + sizeof(int32_t));
  L.rep = off; off = align256(off + sizeof(ebv_refine_report_t));
  L.ws = off;
  L.ws_bytes = std::max(dense_factor_ws(n, prec), dense_solve_ws(n, nrhs, prec));
  off = align256(off + L.ws_bytes);
  L.total = off;
  return L;
}

bool mixed(ebv_prec_t p) { return p == EBV_MIXED_BF16 || p == EBV_MIXED_FP16; }

// Columns [c0, c1) of A from device-accessible (page-locked) host memory into
// the FP64 device copy and the FP32 working copy of the mixed factorisation,
// with its scan words (largest off-diagonal, smallest diagonal magnitude).
// The SMs read host memory directly: strided column blocks copied this way
// run at the host link's rate, twice what 2-D copy-engine transfers reach.
__global__ void k_copy_block(const double *src, int64_t lds, double *a_dev, float *lowp, int64_t n, int64_t c0,
                             int64_t c1, unsigned int *maxoff, unsigned int *mindiag) {
  unsigned int lmax = 0u, lmin = 0x7F800000u;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    const double *srow = src + i * lds;
    double *drow = a_dev + i * n;
    float *wrow = lowp + i * n;
    for (int64_t j = c0 + threadIdx.x; j < c1; j += blockDim.x) {
      const double v = srow[j];
      drow[j] = v;
      const float f = (float)v;
      wrow[j] = f;
      const unsigned int bits = __float_as_uint(fabsf(f));
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

}  // namespace
}  // namespace ebv

using namespace ebv;

extern "C" size_t ebv_gesv_host_workspace_size(const ebv_desc_t *desc, ebv_prec_t prec, int64_t nrhs) {
  if (!desc || desc->n < 0 || nrhs < 0 || desc->storage != EBV_DENSE || !mixed(prec)) return 0;
  return host_layout(desc->n, nrhs, prec).total;
}

extern "C" ebv_status_t ebv_gesv_host(const ebv_desc_t *desc, ebv_prec_t prec, const double *a_host,
                                      const double *b_host, double *x_host, int64_t nrhs, int64_t ldb,
                                      const ebv_refine_t *refine,
                                      ebv_refine_report_t *report_host, int32_t *info_host, void *ws,
                                      size_t ws_bytes, ebv_stream_t stream) {
  if (!desc || desc->storage != EBV_DENSE) return EBV_ERR_ARG;
  if (!mixed(prec)) return EBV_ERR_UNSUPPORTED;
  const int64_t n = desc->n;
  if (n < 0 || desc->ld < std::max<int64_t>(1, n) || nrhs < 0 || nrhs > (int64_t(1) << 20) ||
      ldb < std::max<int64_t>(1, nrhs))
    return EBV_ERR_ARG;
  if (refine && (!(refine->tol >= 0.0) || refine->max_iter < 0 || refine->max_iter > 1000)) return EBV_ERR_ARG;
  if (n > 0 && (!a_host || (nrhs > 0 && (!b_host || !x_host)))) return EBV_ERR_ARG;
  const HostLayout L = host_layout(n, nrhs, prec);
  if (!ws || (uintptr_t)ws % 256 != 0 || ws_bytes < L.total) return EBV_ERR_WORKSPACE;
  if (n == 0) return EBV_OK;
  cudaStream_t s = (cudaStream_t)stream;
  char *w = (char *)ws;
  double *a_dev = (double *)(w + L.a);
  float *lowp = (float *)(w + L.lowp);
  double *x_dev = (double *)(w + L.x);
  int32_t *info_dev = (int32_t *)(w + L.info);
  ebv_refine_report_t *rep_dev = (ebv_refine_report_t *)(w + L.rep);
  void *fws = w + L.ws;
  HostPipe *p = nullptr;
  EBV_TRY(host_pipe(&p));
  // Column blocks: at least 1024 columns, at most kMaxCopyBlocks of them.
  const int64_t cbw = std::max<int64_t>(1024, ((n + kMaxCopyBlocks - 1) / kMaxCopyBlocks + 63) / 64 * 64);
  const int nb = ceil_div(n, cbw);
  // Page-locked A is read by a copy kernel that also writes the FP32 working
  // copy; other host memory goes through 2-D copies and the factorisation
  // converts each block itself.
  cudaPointerAttributes attr{};
  const bool direct = cudaPointerGetAttributes(&attr, a_host) == cudaSuccess && attr.type == cudaMemoryTypeHost &&
                      attr.devicePointer != nullptr;
  if (!direct) (void)cudaGetLastError();  // an unregistered pointer is not an error here
  unsigned int *scan = nullptr;
  if (direct) {
    static const cudaError_t carveout = set_smem(k_copy_block, 0);
    if (carveout != cudaSuccess) return EBV_ERR_CUDA;
    scan = dense_factor_scan_init(n, prec, fws, s);
    if (!scan) return EBV_ERR_CUDA;
  }
  // Copies on the pipe's stream, after everything already queued on `stream`.
  EBV_CU(cudaEventRecord(p->fork, s));
  EBV_CU(cudaStreamWaitEvent(p->cs, p->fork, 0));
  for (int b = 0; b < nb; ++b) {
    const int64_t c0 = (int64_t)b * cbw, c1 = std::min<int64_t>(n, c0 + cbw);
    if (direct) {
      k_copy_block<<<(int)std::min<int64_t>(n, 128), 256, 0, p->cs>>>((const double *)attr.devicePointer, desc->ld,
                                                                       a_dev, lowp, n, c0, c1, scan, scan + 1);
      EBV_TRY(launch_ok());
    } else {
      EBV_CU(cudaMemcpy2DAsync(a_dev + c0, (size_t)n * 8, a_host + c0, (size_t)desc->ld * 8, (size_t)(c1 - c0) * 8,
                               (size_t)n, cudaMemcpyHostToDevice, p->cs));
    }
    EBV_CU(cudaEventRecord(p->ev[b], p->cs));
  }
  if (nrhs > 0)
    EBV_CU(cudaMemcpy2DAsync(x_dev, (size_t)nrhs * 8, b_host, (size_t)ldb * 8, (size_t)nrhs * 8, (size_t)n,
                             cudaMemcpyHostToDevice, p->cs));
  EBV_CU(cudaEventRecord(p->ev[kMaxCopyBlocks], p->cs));
  EBV_TRY(dense_factor_staged(n, prec, a_dev, lowp, info_dev, fws, L.ws_bytes, p->ev, cbw, !direct, s));
  EBV_CU(cudaStreamWaitEvent(s, p->ev[kMaxCopyBlocks], 0));  // B is there; the copy stream joins back
  if (nrhs > 0) {
    ebv_desc_t dd = *desc;
    dd.ld = n;
    EBV_TRY(ebv_solve(&dd, prec, lowp, a_dev, x_dev, nrhs, nrhs, refine, refine ? rep_dev : nullptr, fws, L.ws_bytes,
                      stream));
    EBV_CU(cudaMemcpy2DAsync(x_host, (size_t)ldb * 8, x_dev, (size_t)nrhs * 8, (size_t)nrhs * 8, (size_t)n,
                             cudaMemcpyDeviceToHost, s));
  }
  if (refine && report_host)
    EBV_CU(cudaMemcpyAsync(report_host, rep_dev, sizeof(ebv_refine_report_t), cudaMemcpyDeviceToHost, s));
  if (info_host) EBV_CU(cudaMemcpyAsync(info_host, info_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  return EBV_OK;
}
