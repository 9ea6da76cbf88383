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

// Shared-memory layout of one CTA of a cluster of nc CTAs (element sizes of the
// storage and of the compute type), identical in every CTA of the cluster: 14
// state slices [3][rb nx] of the storage type (y_n, k_1..k_7, two stage states,
// the stage-7 error sum, the demagnetising field), then (complex) the
// x-transformed rows [3 rb][Kx], the y-inverse-transformed columns [3 cb][ny],
// the y spectra of the CTA's columns [3 cb][Py], the two half-length inverses
// of 64-point columns [3 cb][2][32], the table W_64^q, and (real) the tensor of
// the CTA's kx columns [4][cb][Py/2 + 1].
struct SmallLayout {
    size_t rows, cols, spec, half, w64, tens, total;    // byte offsets and the total
};
__host__ __device__ inline SmallLayout small_layout(const SimDesc& d, int nc, size_t ssz, size_t csz) {
    const int rb = small_rows_per_cta(d, nc), cb = small_cols_per_cta(d, nc);
    const size_t z = 2 * csz;
    SmallLayout L;
    size_t b = ((14 * 3 * (size_t)rb * d.nx * ssz) + 15) & ~(size_t)15;
    L.rows = b;
    b += 3 * (size_t)rb * d.Kx * z;
    L.cols = b;
    b += 3 * (size_t)cb * d.ny * z;
    L.spec = b;
    b += 3 * (size_t)cb * d.Py * z;
    L.half = b;
    b += (d.Py == 64 ? 3 * (size_t)cb * 64 : 0) * z;
    L.w64 = b;
    b += 64 * z;
    L.tens = b;
    b += 4 * (size_t)cb * (d.Py / 2 + 1) * csz;
    L.total = (b + 15) & ~(size_t)15;
    return L;
}
inline size_t small_smem_bytes(const SimDesc& d, int nc, size_t ssz, size_t csz) {
    return small_layout(d, nc, ssz, csz).total;
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
