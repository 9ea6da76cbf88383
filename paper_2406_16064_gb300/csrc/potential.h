// Host interface of the scalar-potential demagnetising field (potential.cu),
// used by the context API (api.cu).
#pragma once
#include <cuda_runtime.h>

namespace mm {

// Padded geometry: P = the smallest power of two >= 2n + 1 per axis (offsets
// -n..n of the potential kernel), Kx = Px / 2 + 1 stored x bins.
struct PotGeom {
    int nx, ny, nz;
    int Px, Py, Pz, lPx, lPy, lPz, Kx;
    double dx, dy, dz;
};

// Largest padded length of the scalar-potential path (one row of Px complex
// FP64 values, twice, in one CTA's shared memory).
constexpr int kPotMaxP = 2048;

// Device buffers of one geometry: the kernel spectrum S^ [3][Pz][Py][Kx]
// (complex, context precision, scaled by 1 / (Px Py Pz)), the magnetisation
// spectrum M^ [3][Pz][Py][Kx], the potential spectrum U [Pz][Py][Kx] and the
// potential u on the mesh extended by one cell on every side.
struct PotBuffers {
    void* Shat = nullptr;
    void* Mhat = nullptr;
    void* U = nullptr;
    void* u = nullptr;
};

PotGeom pot_geometry(int nx, int ny, int nz, double dx, double dy, double dz);
long long pot_bins(const PotGeom& g);        // Pz Py Kx
long long pot_ext_cells(const PotGeom& g);   // (nx + 2)(ny + 2)(nz + 2)
// S^ in FP64 (scratch64: 3 pot_bins complex doubles), stored in Shat (FP32 or FP64)
cudaError_t pot_precompute(cudaStream_t s, const PotGeom& g, void* Shat, bool f32, void* scratch64, const void* twd,
                           long long* launches);
// H_d of m (context precision, [3][N]); Ms: per-cell array or NULL for Msu
cudaError_t pot_field(cudaStream_t s, const PotGeom& g, const PotBuffers& B, bool f32, const void* m,
                      const void* Ms, double Msu, void* H, const void* tw, long long* launches);

}  // namespace mm
