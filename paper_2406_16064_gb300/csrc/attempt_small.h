// Host interface of the single-launch Dormand-Prince attempts of small
// single-plane meshes (attempt_small.cu), used by the context API (api.cu).
#pragma once
#include <cuda_runtime.h>

#include "mm_kernels.cuh"

namespace mm {

// Largest padded FFT length along x and y of the single-launch path (meshes of
// at most 32 x 32 cells), and the largest cluster it runs on.
constexpr int kSmallMaxP = 64;
constexpr int kSmallMaxCluster = 16;
constexpr int kSmallThreads = 256;

// A simulation the single-launch path can run: one plane, padded lengths within
// kSmallMaxP, no extended terms, not a NEB chain member.
inline bool small_eligible(const SimDesc& d) {
    return d.nz == 1 && d.Pz == 1 && d.Px <= kSmallMaxP && d.Py <= kSmallMaxP && (d.flags & F_EXT) == 0 &&
           d.group_begin < 0;
}

// Rows and kx columns of one CTA for a cluster of nc CTAs: CTA b owns rows
// [b rb, min(ny, (b + 1) rb)) and kx columns [b cb, min(Kx, (b + 1) cb)).
__host__ __device__ inline int small_rows_per_cta(const SimDesc& d, int nc) { return (d.ny + nc - 1) / nc; }
__host__ __device__ inline int small_cols_per_cta(const SimDesc& d, int nc) { return (d.Kx + nc - 1) / nc; }

// Dynamic shared memory of one CTA (element sizes of the storage and of the
// compute type): 13 state slices [3][rb nx] (y_n, k_1..k_7, two stage states,
// the stage-7 error sum), then two row buffers of 3 rb padded sequences of Kx
// complex values and two column buffers of 3 cb padded sequences of Py.
inline size_t small_smem_bytes(const SimDesc& d, int nc, size_t ssz, size_t csz) {
    const int rb = small_rows_per_cta(d, nc), cb = small_cols_per_cta(d, nc);
    size_t b = ((13 * 3 * (size_t)rb * d.nx * ssz) + 15) & ~(size_t)15;
    b += 2 * 3 * (size_t)rb * padded_len(d.Kx) * 2 * csz;
    b += 2 * 3 * (size_t)cb * padded_len(d.Py) * 2 * csz;
    return b;
}

struct SmallLaunch {
    cudaStream_t stream = nullptr;
    const SimDesc* desc = nullptr;     // device descriptors of the batch
    SimState* state = nullptr;         // device integration state
    int nsims = 0;
    void* m = nullptr;                 // batch state (storage type)
    const void* tensor = nullptr;      // stored tensor (compute type)
    const void* Ms = nullptr;          // per-cell Ms (storage type)
    const void* tw = nullptr;          // twiddle tables (compute type)
    int kind = 0;                      // 0 FP32, 1 FP64 native, 2 FP64 storage with double-float transforms
    int cluster = 0;                   // CTAs per simulation
    size_t smem = 0;                   // dynamic shared memory per CTA
    int n_attempts = 0;
};

// Whether the device can co-schedule a cluster of nc CTAs of this kind with
// `smem` bytes of dynamic shared memory each.
bool small_cluster_fits(int kind, size_t smem, int nc);
// Issue one launch that runs n_attempts attempts of every simulation.
cudaError_t small_attempts(const SmallLaunch& L);

}  // namespace mm
