// Single-launch Dormand-Prince attempts (attempt_small.cuh) for MM_F64_NATIVE contexts: FP64 arithmetic throughout.
#include "attempt_small.cuh"

namespace mm {
bool small_fits_f64(size_t smem, int nc) { return small_fits_t<double>(smem, nc); }
cudaError_t small_launch_f64(const SmallLaunch& L) { return small_launch_t<double>(L); }
}  // namespace mm
