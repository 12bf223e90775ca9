// Adjoint (placeholder entry point).
#include "common.cuh"

extern "C" ebv_status_t ebv_solve_adjoint(int64_t, int64_t, int64_t, const double *, int64_t, int64_t,
                                          const double *, const double *, double *, double *, ebv_stream_t) {
  return EBV_ERR_UNSUPPORTED;
}
