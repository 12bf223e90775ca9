// Batched factor + solve (placeholder entry points).
#include "common.cuh"
#include "internal.h"

extern "C" {
int64_t ebv_batch_schedule_len(int64_t batch) { return batch < 0 ? 0 : 2 * batch + 8; }
size_t ebv_batch_workspace_size(int64_t) { return ebv::kStatusBytes; }
ebv_status_t ebv_batch_schedule(int64_t, const int32_t *, const int32_t *, const int8_t *, int32_t *) {
  return EBV_ERR_UNSUPPORTED;
}
ebv_status_t ebv_factor_solve_batched(int64_t, const int32_t *, const int32_t *, void *const *, void *const *,
                                      ebv_prec_t, const int32_t *, int32_t *, void *, size_t, ebv_stream_t) {
  return EBV_ERR_UNSUPPORTED;
}
size_t ebv_batch_autotune_scratch(int32_t, int32_t, ebv_prec_t) { return 0; }
ebv_status_t ebv_batch_autotune(const int32_t *, int32_t, int32_t, ebv_prec_t, void *, size_t, int8_t *, float *,
                                ebv_stream_t) {
  return EBV_ERR_UNSUPPORTED;
}
}
