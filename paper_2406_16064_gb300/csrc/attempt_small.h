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

// Rows and column units of one CTA for a cluster of nc CTAs.  A column unit is
// one kx column (Py <= 32) or one half of it (Py = 64: the even and the odd ky
// bins, each a 32-point transform): unit u = kx H + hf, H = 1 or 2.  CTA b owns
// rows [b rb, min(ny, (b + 1) rb)) and units [b cu, min(Kx H, (b + 1) cu)).
__host__ __device__ inline int small_halves(const SimDesc& d) { return d.Py == 64 ? 2 : 1; }
__host__ __device__ inline int small_rows_per_cta(const SimDesc& d, int nc) { return (d.ny + nc - 1) / nc; }
__host__ __device__ inline int small_units_per_cta(const SimDesc& d, int nc) {
    return (d.Kx * small_halves(d) + nc - 1) / nc;
}

// Row of a column unit's spectrum in shared memory: bin k at k + k/8, so the
// bit-reversed stores of a warp spread over the banks.
__host__ __device__ inline int small_spec_row(int lyh) { return lyh + lyh / 8 + 1; }

// Shared-memory layout of one CTA (element sizes of the storage and of the
// compute type), identical in every CTA of the cluster: 14 state slices
// [3][rb nx] of the storage type (y_n, k_1..k_7, two stage states, the stage-7
// error sum, the demagnetising field) and the halo rows [2][2][3][nx] (the rows
// below and above the CTA's block, by stage-state parity), then (complex) the
// rows pushed to the CTA's column units [3 cu][ny], the units' spectra
// [3 cu][small_spec_row(Py / H)], the column results pushed to the CTA's rows [3 rb][Kx][H],
// the table W_64^q, and (real) the tensor at the units' bins [4][cu][Py / H].
struct SmallLayout {
    size_t halo, colin, spec, rowin, w64, tens, total;    // byte offsets and the total
};
__host__ __device__ inline SmallLayout small_layout(const SimDesc& d, int nc, size_t ssz, size_t csz) {
    const int rb = small_rows_per_cta(d, nc), cu = small_units_per_cta(d, nc), H = small_halves(d);
    const int lyh = d.Py / H;
    const size_t z = 2 * csz;
    SmallLayout L;
    size_t b = 14 * 3 * (size_t)rb * d.nx * ssz;
    L.halo = b;
    b += 2 * 2 * 3 * (size_t)d.nx * ssz;
    b = (b + 15) & ~(size_t)15;
    L.colin = b;
    b += 3 * (size_t)cu * d.ny * z;
    L.spec = b;
    b += 3 * (size_t)cu * small_spec_row(lyh) * z;
    L.rowin = b;
    b += 3 * (size_t)rb * d.Kx * H * z;
    L.w64 = b;
    b += 64 * z;
    L.tens = b;
    b += 4 * (size_t)cu * lyh * csz;
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
