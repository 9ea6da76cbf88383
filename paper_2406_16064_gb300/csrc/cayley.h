// Host interface of the fixed-step RK4 integrators (cayley.cu), used by the
// context API (api.cu).
#pragma once
#include <cuda_runtime.h>

#include "engine.cuh"

namespace mm {

struct Rk4Buffers {
    void* m = nullptr;      // state m_n, updated in place
    void* ys = nullptr;     // stage state
    void* H = nullptr;      // Cayley: effective field at the stage state
    void* dmdt = nullptr;   // Cayley: scratch for the right-hand side the field passes also write
    void* k[4] = {};        // stage slopes: dm/dt (projection) or d omega/dt (Cayley)
};

// One RK4 step of size h (seconds) of every simulation, projected or on the
// Cayley variable; advances each simulation's time by h.  No synchronisation.
template <typename T>
void rk4_step(const Launch& L, const Rk4Buffers& B, double h, bool cayley);

}  // namespace mm
