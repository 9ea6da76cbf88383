// Host-side engine interface: issues the kernels of one right-hand side, of
// one Dormand-Prince attempt, or of one NEB attempt, for a whole batch (or a
// single simulation) on a stream.  Instantiated for float and double in
// engine_f32.cu / engine_f64.cu.
#pragma once
#include <cuda_runtime.h>

#include "mm_kernels.cuh"

namespace mm {

struct ItemSet {
    const WorkItem* dev = nullptr;
    int count = 0;
};

// Kernel kinds reported by the profiling hook.
enum { KIND_XFWD = 0, KIND_YFWD, KIND_ZCOL, KIND_YINV, KIND_YFUSED, KIND_XINV, KIND_CONTROL, KIND_PROJECT,
       KIND_NEB, KIND_YZC, KIND_COUNT };

// Records a CUDA event on the launch stream after every kernel; the interval
// between consecutive events is attributed to the kernel that ended it.
struct ProfileHook {
    cudaStream_t stream = nullptr;
    cudaEvent_t* ev = nullptr;
    int* kinds = nullptr;
    int cap = 0, used = 0;
    void mark(int kind) {
        if (used < cap) {
            cudaEventRecord(ev[used], stream);
            kinds[used] = kind;
            ++used;
        }
    }
};

struct Launch {
    cudaStream_t stream = nullptr;
    const SimDesc* desc = nullptr;
    SimState* state = nullptr;
    int nsims = 0;
    ItemSet x, y13, z, y2;        // x rows, y fwd/inv (nz > 8), z fused, y fused (films)
    ItemSet cell;                 // per-cell tiles of ~kCellTile cells (NEB tangent and force)
    ItemSet yzc[kYzcListCount];   // cluster-fused y/z, one list per plane count, groups, CTAs per SM
    size_t smem_x = 0, smem_xi = 0, smem_y13 = 0, smem_z = 0, smem_y2 = 0, smem_yzc = 0;
    int x_threads = 0, col_threads = 0;   // tuned CTA widths of the x and column passes (0: rule)
    bool dd = false;              // FP64 storage with double-float transforms (tensor, spectrum, tw in dd)
    const void* tensor = nullptr;
    const void* Ms = nullptr;
    const void* cellp = nullptr;  // per-cell A and D blocks
    bool ext = false;             // some simulation has extended terms (F_EXT)
    const void* tw = nullptr;
    void* spec = nullptr;
    long long* launches = nullptr;
    ProfileHook* hook = nullptr;
};

struct RkBuffers {
    void* m = nullptr;
    void* ybuf = nullptr;
    void* const* kvec_dev = nullptr;   // device array of the 7 k pointers
    void* kvec[7] = {};
    void* errp = nullptr;
    void* heff = nullptr;              // NEB: effective field of every image
    void* tau = nullptr;               // NEB: tangents
};

template <typename T>
void engine_rhs(const Launch& L, int mode, const T* m, T* dmdt, T* heff, long long off_adjust);
// FP64 storage, double-float transforms (engine_dd.cu)
void engine_rhs_dd(const Launch& L, int mode, const double* m, double* dmdt, double* heff, long long off_adjust);
void engine_attempt_dd(const Launch& L, const RkBuffers& B);
void engine_neb_attempt_dd(const Launch& L, const RkBuffers& B);
template <typename T>
void engine_attempt(const Launch& L, const RkBuffers& B);
template <typename T>
void engine_neb_attempt(const Launch& L, const RkBuffers& B);
void engine_set_attributes();
void engine_bounded_wait(cudaStream_t s, int* flag, long long spins, int* status);
void engine_after_stage1(const Launch& L);

// newell.cu
void upload_gauss_legendre();
// FP64, FP32 and double-float (hi, lo pairs of the FP64 values) twiddle tables
void launch_twiddles(cudaStream_t s, void* twd, void* twf, void* twdd);
void launch_newell_octant(cudaStream_t s, int nx, int ny, int nz, double dx, double dy, double dz, double* oct);
void launch_newell_place(cudaStream_t s, const double* oct, int c, int nx, int ny, int nz, int Px, int Py, int Pz,
                         void* buf);
void launch_fft_axis_f64(cudaStream_t s, void* buf, int Px, int Py, int Pz, int axis, const void* twd);
// Ty > 0: the blocked layout of the cluster-fused y/z pass with qp values per bin;
// nk: kz bins (Pz/2+1) or, for the cluster pass, the nz dz planes of an x-y
// transformed buffer (imag_xz: xz and yz are imaginary there)
// out_kind: 0 FP64, 1 FP32, 2 double-float (hi, lo FP32 pairs)
void launch_newell_extract(cudaStream_t s, const void* buf, int c, int Px, int Py, int Kx, int Pyh, int nk,
                           double scale, void* out, int out_kind, int Ty, int qp, int imag_xz,
                           unsigned long long* maxim, unsigned long long* maxre);

}  // namespace mm
