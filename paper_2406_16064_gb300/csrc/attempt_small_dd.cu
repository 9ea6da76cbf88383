// Single-launch Dormand-Prince attempts (attempt_small.cuh) for MM_F64 contexts: FP64 state, prologue and epilogue, transforms in double-float.
#include "attempt_small.cuh"

namespace mm {
bool small_fits_dd(size_t smem, int nc) { return small_fits_t<dd>(smem, nc); }
cudaError_t small_launch_dd(const SmallLaunch& L) { return small_launch_t<dd>(L); }
}  // namespace mm
