// mm_rhs_eval_static: the right-hand-side evaluation of one simulation for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside a host callback or
// a tightly budgeted embedding (a plugin handed a device pointer by its host
// application, a process whose allocator is owned by someone else) may only
// launch work on memory it was given.  For them this entry point allocates
// nothing.  The caller passes the state and the output buffers; every
// intermediate (twiddle tables, the FP64 Newell octant and its FFT buffer, the
// stored tensor spectrum, the demag spectrum, the descriptor and work lists)
// lives in one file-scope __device__ array of MM_STATIC_SCRATCH_BYTES.  Every
// GPU that loads libmm holds that array until the process exits.
//
// The first call on a device looks up the array's device address with
// cudaGetSymbolAddress (host code cannot use the symbol itself: in host code it
// names a host-side shadow, not device memory); make that first call before any
// stream capture.  All calls share the array and it keeps the last call's
// contents, so calls that overlap on the GPU (different streams, or host
// threads) race: serialise them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "engine.cuh"
#include "mm.h"

using namespace mm;

#define MM_STATIC_SCRATCH_BYTES (32u << 20)   // 32 MiB
#define MM_STATIC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_static_scratch[MM_STATIC_SCRATCH_BYTES];

void mm_internal_set_error(const char* msg);   // api.cu

namespace {

std::mutex g_lock;
void* g_base[MM_STATIC_MAX_DEVICES] = {};

int err(int code, const char* msg) {
    mm_internal_set_error(msg);
    return code;
}

int lg2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

int padded(int n, bool min2) {
    if (n <= 1) return min2 ? 2 : 1;
    int p = 1;
    while (p < 2 * n - 1) p <<= 1;
    return p;
}

int floor2(int v) {
    int p = 1;
    while (p * 2 <= v) p *= 2;
    return p;
}

// bump allocator over the static array (offsets only)
struct Carve {
    size_t used = 0;
    size_t take(size_t bytes) {
        const size_t at = (used + 255) & ~size_t(255);
        used = at + bytes;
        return at;
    }
};

}  // namespace

extern "C" int mm_rhs_eval_static(const mm_mesh* mesh, const mm_material* mat, int precision,
                                  const void* m_dev, void* dmdt_dev, void* heff_dev, void* cuda_stream) {
    if (!mesh || !mat || !m_dev || !dmdt_dev) return err(MM_EINVAL, "mm_rhs_eval_static: NULL argument");
    if (precision != MM_F64 && precision != MM_F32) return err(MM_EINVAL, "mm_rhs_eval_static: bad precision");
    if (mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1 || !(mesh->dx > 0 && mesh->dy > 0 && mesh->dz > 0))
        return err(MM_EINVAL, "mm_rhs_eval_static: bad mesh");
    if (!(mat->Ms >= 0) || !(mat->alpha >= 0) || !(mat->gamma > 0))
        return err(MM_EINVAL, "mm_rhs_eval_static: bad material");
    if (mat->dmi_kind != MM_DMI_NONE && mat->dmi_kind != MM_DMI_INTERFACIAL)
        return err(MM_EINVAL, "mm_rhs_eval_static: unsupported DMI kind");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const bool f32 = precision == MM_F32;
    const size_t e = f32 ? 4 : 8;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MM_STATIC_MAX_DEVICES)
        return err(MM_ECUDA, "mm_rhs_eval_static: no current CUDA device");
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_base[dev]) {
        void* p = nullptr;
        const cudaError_t rc = cudaGetSymbolAddress(&p, g_static_scratch);
        if (rc != cudaSuccess || !p) return err(MM_ECUDA, "mm_rhs_eval_static: cudaGetSymbolAddress failed");
        g_base[dev] = p;
    }
    unsigned char* base = (unsigned char*)g_base[dev];

    // descriptor of the single simulation (same layout rules as a context)
    SimDesc d;
    memset(&d, 0, sizeof(d));
    d.nx = mesh->nx; d.ny = mesh->ny; d.nz = mesh->nz;
    const long long n = (long long)d.nx * d.ny * d.nz;
    if (n > (1LL << 26)) return err(MM_EINVAL, "mm_rhs_eval_static: mesh too large for the static scratch");
    d.ncells = (int)n;
    d.Px = padded(d.nx, true); d.Py = padded(d.ny, false); d.Pz = padded(d.nz, false);
    const int lim = f32 ? 8192 : 4096;
    if (d.Px > 8192 || d.Py > lim || d.Pz > lim) return err(MM_EINVAL, "mm_rhs_eval_static: padded FFT too long");
    d.lPx = lg2(d.Px); d.lPy = lg2(d.Py); d.lPz = lg2(d.Pz);
    d.Kx = d.Px / 2 + 1; d.Pyh = d.Py / 2 + 1; d.Pzh = d.Pz / 2 + 1;
    d.ncomp = d.Pz > 1 ? 6 : 4;
    const double un = sqrt(mat->u[0] * mat->u[0] + mat->u[1] * mat->u[1] + mat->u[2] * mat->u[2]);
    if (mat->Ku != 0.0 && !(un > 0)) return err(MM_EINVAL, "mm_rhs_eval_static: anisotropy axis is zero");
    for (int i = 0; i < 3; ++i) { d.u[i] = un > 0 ? mat->u[i] / un : 0.0; d.H[i] = mat->H[i]; }
    d.Ms = mat->Ms; d.A = mat->A; d.D = mat->D; d.Ku = mat->Ku; d.Kc = mat->Kc;
    d.alpha = mat->alpha; d.gamma = mat->gamma;
    d.dx = mesh->dx; d.dy = mesh->dy; d.dz = mesh->dz;
    d.flags = (mat->demag ? F_DEMAG : 0) | (mat->dmi_kind == MM_DMI_INTERFACIAL ? F_DMI : 0) |
              (mat->precession ? F_PREC : 0);
    d.group_begin = d.group_end = -1;
    d.neb_index = -1;
    d.ms_off = -1;
    d.off = 0;
    d.spec_off = 0;
    d.tens_off = 0;
    const int EB = f32 ? 4096 : 2048;
    const int rows = d.ny * d.nz;
    d.Rx = std::max(1, std::min(rows, EB / d.Kx));
    const int kcap = std::min(32, 1 << lg2(d.Kx));
    d.Ty = std::min(kcap, floor2(std::max(1, (d.Pz > 1 ? 3 : 1) * EB / d.Py)));
    d.Tz = std::min(kcap, floor2(std::max(1, EB / d.Pz)));
    const bool demag = mat->demag != 0;
    std::vector<WorkItem> xv, y13v, zv, y2v;
    for (int r0 = 0; r0 < rows; r0 += d.Rx) xv.push_back({0, r0, std::min(d.Rx, rows - r0), 0});
    if (demag) {
        if (d.Pz > 1) {
            if (d.Py > 1)
                for (int z = 0; z < d.nz; ++z)
                    for (int k0 = 0; k0 < d.Kx; k0 += d.Ty)
                        for (int c = 0; c < 3; ++c) y13v.push_back({0, z, k0, c});
            for (int ky = 0; ky < d.Py; ++ky)
                for (int k0 = 0; k0 < d.Kx; k0 += d.Tz) zv.push_back({0, ky, k0, 0});
        } else if (d.Py > 1) {
            for (int k0 = 0; k0 < d.Kx; k0 += d.Ty) y2v.push_back({0, 0, k0, -1});
        }
    }
    const size_t vsz = 2 * e;
    const size_t smem_x = 3 * (size_t)d.Rx * d.Kx * vsz;
    const size_t smem_y13 = (size_t)d.Py * d.Ty * vsz;
    const size_t smem_y2 = 3 * (size_t)d.Py * d.Ty * vsz;
    const size_t smem_z = 3 * (size_t)d.Pz * d.Tz * vsz;
    if (smem_x > 227 * 1024 - 4096 || smem_y13 > 227 * 1024 || smem_y2 > 227 * 1024 || smem_z > 227 * 1024)
        return err(MM_EINVAL, "mm_rhs_eval_static: FFT tile exceeds shared memory");

    // carve the static array
    Carve cv;
    const size_t o_twd = cv.take((size_t)MM_LMAX * 16);
    const size_t o_twf = cv.take((size_t)MM_LMAX * 8);
    const size_t o_desc = cv.take(sizeof(SimDesc));
    const size_t o_state = cv.take(sizeof(SimState));
    const size_t o_diag = cv.take(2 * sizeof(unsigned long long));
    const size_t o_xi = cv.take(std::max<size_t>(1, xv.size()) * sizeof(WorkItem));
    const size_t o_y13 = cv.take(std::max<size_t>(1, y13v.size()) * sizeof(WorkItem));
    const size_t o_z = cv.take(std::max<size_t>(1, zv.size()) * sizeof(WorkItem));
    const size_t o_y2 = cv.take(std::max<size_t>(1, y2v.size()) * sizeof(WorkItem));
    const long long tens_elems = (long long)d.ncomp * d.Pzh * d.Pyh * d.Kx;
    const long long spec_elems = demag ? 3LL * d.nz * d.Py * d.Kx : 0;
    const size_t o_tens = cv.take(demag ? (size_t)tens_elems * e : 16);
    const size_t o_spec = cv.take(demag ? (size_t)spec_elems * vsz : 16);
    const size_t o_oct = cv.take(demag ? (size_t)6 * n * 8 : 16);
    const size_t o_fft = cv.take(demag ? (size_t)d.Px * d.Py * d.Pz * 16 : 16);
    if (cv.used > MM_STATIC_SCRATCH_BYTES)
        return err(MM_EINVAL, "mm_rhs_eval_static: mesh needs more than the 32 MiB static scratch "
                              "(padded FFT grid, Newell octant, tensor and spectrum)");

#define SCK(x)                                                                         \
    do {                                                                               \
        if ((x) != cudaSuccess) return err(MM_ECUDA, "mm_rhs_eval_static: " #x);       \
    } while (0)
    SCK(cudaMemcpyAsync(base + o_desc, &d, sizeof(d), cudaMemcpyHostToDevice, s));
    SCK(cudaMemsetAsync(base + o_state, 0, sizeof(SimState), s));
    SCK(cudaMemsetAsync(base + o_diag, 0, 2 * sizeof(unsigned long long), s));
    auto up = [&](size_t off, const std::vector<WorkItem>& v) {
        return v.empty() ? cudaSuccess
                         : cudaMemcpyAsync(base + off, v.data(), v.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, s);
    };
    SCK(up(o_xi, xv));
    SCK(up(o_y13, y13v));
    SCK(up(o_z, zv));
    SCK(up(o_y2, y2v));
    launch_twiddles(s, base + o_twd, base + o_twf);
    upload_gauss_legendre();
    engine_set_attributes();
    SCK(cudaGetLastError());

    if (demag) {
        double* oct = (double*)(base + o_oct);
        void* fftbuf = base + o_fft;
        launch_newell_octant(s, d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, oct);
        const double scale = 1.0 / ((double)d.Px * d.Py * d.Pz);
        unsigned long long* diag = (unsigned long long*)(base + o_diag);
        for (int c = 0; c < d.ncomp; ++c) {
            launch_newell_place(s, oct, c, d.nx, d.ny, d.nz, d.Px, d.Py, d.Pz, fftbuf);
            for (int ax = 0; ax < 3; ++ax) launch_fft_axis_f64(s, fftbuf, d.Px, d.Py, d.Pz, ax, base + o_twd);
            launch_newell_extract(s, fftbuf, c, d.Px, d.Py, d.Kx, d.Pyh, d.Pzh, scale, base + o_tens, f32, diag,
                                  diag + 1);
        }
        SCK(cudaGetLastError());
        unsigned long long hb[2];
        SCK(cudaMemcpyAsync(hb, diag, sizeof(hb), cudaMemcpyDeviceToHost, s));
        SCK(cudaStreamSynchronize(s));
        double im, re;
        memcpy(&im, &hb[0], 8);
        memcpy(&re, &hb[1], 8);
        if (re > 0 && !(im / re < 1e-9)) return err(MM_ECUDA, "mm_rhs_eval_static: tensor spectrum not real");
    }

    Launch L;
    L.stream = s;
    L.desc = (const SimDesc*)(base + o_desc);
    L.state = (SimState*)(base + o_state);
    L.nsims = 1;
    L.x = {(const WorkItem*)(base + o_xi), (int)xv.size()};
    L.y13 = {(const WorkItem*)(base + o_y13), (int)y13v.size()};
    L.z = {(const WorkItem*)(base + o_z), (int)zv.size()};
    L.y2 = {(const WorkItem*)(base + o_y2), (int)y2v.size()};
    L.smem_x = smem_x;
    L.smem_y13 = y13v.empty() ? 0 : smem_y13;
    L.smem_z = zv.empty() ? 0 : smem_z;
    L.smem_y2 = y2v.empty() ? 0 : smem_y2;
    L.tensor = base + o_tens;
    L.Ms = nullptr;
    L.tw = f32 ? (const void*)(base + o_twf) : (const void*)(base + o_twd);
    L.spec = base + o_spec;
    if (f32)
        engine_rhs<float>(L, MODE_RHS, (const float*)m_dev, (float*)dmdt_dev, (float*)heff_dev, 0);
    else
        engine_rhs<double>(L, MODE_RHS, (const double*)m_dev, (double*)dmdt_dev, (double*)heff_dev, 0);
    SCK(cudaGetLastError());
#undef SCK
    return MM_OK;
}
