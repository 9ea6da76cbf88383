// Host interface of the steepest-descent minimiser (minimize.cu), used by the
// context API (api.cu).
#pragma once
#include <cuda_runtime.h>

#include "engine.cuh"

namespace mm {

// Per-simulation state of the minimiser (device array, one per simulation).
struct SdState {
    double tau;                    // step size tau_k (m/A)
    double ss, sy, yy;             // sums over the cells of s.s, s.y, y.y
    double dmdt_scale;             // |dm/dt| / |g| of the material's LL right-hand side
    double stop_dmdt;              // stop once max |dm/dt| < stop_dmdt (rad/s; 0 = never)
    double max_dmdt;               // max |dm/dt| at the last step's m, rad/s
    unsigned long long maxg_bits;  // max |g|^2 over the cells (ordered bits)
    long long k;                   // steps taken
    int status;                    // 0 running, 2 converged, -4 non-finite
    int pad;
};

struct SdBuffers {
    void* m = nullptr;      // state m_k, updated in place
    void* H = nullptr;      // effective field at m_k
    void* dmdt = nullptr;   // scratch: the right-hand side the field passes also write
    void* mprev = nullptr;  // m_{k-1}
    void* gprev = nullptr;  // g_{k-1}, then g_k
    SdState* sd = nullptr;
};

// One step of every running simulation: the effective field, the reductions,
// the step size and the update (four to six launches, no synchronisation).
template <typename T>
void sd_step(const Launch& L, const SdBuffers& B);

}  // namespace mm
