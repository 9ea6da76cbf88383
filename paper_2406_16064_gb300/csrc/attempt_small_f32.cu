// Single-launch Dormand-Prince attempts (attempt_small.cuh) for FP32 contexts: state and arithmetic in FP32.
#include "attempt_small.cuh"

namespace mm {
bool small_fits_f32(size_t smem, int nc) { return small_fits_t<float>(smem, nc); }
cudaError_t small_launch_f32(const SmallLaunch& L) { return small_launch_t<float>(L); }

bool small_fits_f64(size_t smem, int nc);
bool small_fits_dd(size_t smem, int nc);
cudaError_t small_launch_f64(const SmallLaunch& L);
cudaError_t small_launch_dd(const SmallLaunch& L);

bool small_cluster_fits(int kind, size_t smem, int nc) {
    if (smem > 227 * 1024 || nc < 1 || nc > kSmallMaxCluster) return false;
    switch (kind) {
        case 0: return small_fits_f32(smem, nc);
        case 1: return small_fits_f64(smem, nc);
        default: return small_fits_dd(smem, nc);
    }
}

cudaError_t small_attempts(const SmallLaunch& L) {
    switch (L.kind) {
        case 0: return small_launch_f32(L);
        case 1: return small_launch_f64(L);
        default: return small_launch_dd(L);
    }
}
}  // namespace mm
