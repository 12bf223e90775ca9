// Launch counting and optional per-kernel-class timing with CUDA events.
//
// Every kernel launch of the library passes through launch_ok() (which bumps
// the launch counter).  When profiling is switched on (ebv_debug_profile),
// the launches of each class are also bracketed by CUDA events recorded on the
// launching stream; ebv_debug_profile_read() synchronises those events and
// returns, per class, the summed device time, launch count and algorithmic
// work (flops or bytes, as declared at the launch site).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace ebv {
namespace prof {

enum Class : int {
  kLowpGemm = 0,   // tensor-core (or SIMT fallback) mixed-precision trailing update
  kSimtGemm = 1,   // working-precision trailing update
  kPanel = 2,      // diagonal-block kernels
  kTrsv = 3,       // block substitutions
  kResidual = 4,   // refinement residual
  kBatched = 5,    // batched persistent kernel
  kAdjoint = 6,    // adjoint kernels
  kOther = 7,
  kTrsm = 8,       // U12 = L11^{-1} A12: tile products and blocked TRSMs
  kL21 = 9,        // L21 = A21 U11^{-1} tile products
  kLeafUpdate = 10,  // two-leaf middle step (U12 and the A22 update in one launch)
  kInverse = 11,   // product-form inverse (leaf inverses, level products, W Z)
  kNumClasses = 12
};

bool enabled();
// Record the start / end of a launch of class `cls` on stream s; `work` is the
// algorithmic flops (or bytes) of that launch.
void begin(cudaStream_t s, int cls);
void end(cudaStream_t s, int cls, double work);
void count_launch();

struct Scope {
  cudaStream_t s;
  int cls;
  double work;
  Scope(cudaStream_t s_, int c, double w) : s(s_), cls(c), work(w) { begin(s, cls); }
  ~Scope() { end(s, cls, work); }
};

}  // namespace prof
}  // namespace ebv
