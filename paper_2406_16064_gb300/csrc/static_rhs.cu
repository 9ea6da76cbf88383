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
// The first call in each CUDA context (one per device for callers of the
// runtime's primary contexts) looks up the array's device address with
// cudaGetSymbolAddress (host code cannot use the symbol itself: in host code it
// names a host-side shadow, not device memory) and remembers it under that
// context's unique id, so a call made in another context -- a context the
// host application created and made current, or the new primary context
// after cudaDeviceReset -- looks the address up again instead of reusing one
// that belongs to a context that no longer applies.  Make that first call in a
// context before any stream capture.  All calls share the array and it keeps
// the last call's contents, so calls that overlap on the GPU (different
// streams, or host threads) race: serialise them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "engine.cuh"
#include "mm.h"
#include "plan.h"

using namespace mm;

#define MM_STATIC_SCRATCH_BYTES (32u << 20)   // 32 MiB
#define MM_STATIC_MAX_CONTEXTS 64              // remembered (context id, address) pairs

static __device__ __align__(256) unsigned char g_static_scratch[MM_STATIC_SCRATCH_BYTES];

void mm_internal_set_error(const char* msg);   // api.cu

namespace {

std::mutex g_lock;

// The array's device address per CUDA context, keyed by the context's unique id
// (cuCtxGetId: never reused within a process, unlike the context handle).
struct CtxAddr {
    unsigned long long id;
    void* base;
};
CtxAddr g_addr[MM_STATIC_MAX_CONTEXTS];
int g_naddr = 0;

// Driver entry points for the current context's id, fetched through the runtime
// (libmm does not link the driver library).  Signatures of cuCtxGetCurrent and
// cuCtxGetId; CUresult 0 is success.
typedef int (*CtxGetCurrentFn)(void** ctx);
typedef int (*CtxGetIdFn)(void* ctx, unsigned long long* id);

bool current_context_id(unsigned long long* id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        looked_up = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (CtxGetCurrentFn)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (CtxGetIdFn)f;
        cudaGetLastError();
    }
    void* ctx = nullptr;
    if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx) return false;
    return get_id(ctx, id) == 0;
}

// Device address of g_static_scratch in the current context (cudaGetSymbolAddress,
// remembered per context id); nullptr on failure.  Call with g_lock held.
void* scratch_base() {
    unsigned long long id = 0;
    const bool have_id = current_context_id(&id);
    if (have_id)
        for (int i = 0; i < g_naddr; ++i)
            if (g_addr[i].id == id) return g_addr[i].base;
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return nullptr;
    }
    if (have_id) {
        // a full table forgets its oldest entry; a forgotten context just looks up again
        if (g_naddr == MM_STATIC_MAX_CONTEXTS) {
            std::memmove(g_addr, g_addr + 1, (MM_STATIC_MAX_CONTEXTS - 1) * sizeof(CtxAddr));
            --g_naddr;
        }
        g_addr[g_naddr++] = {id, p};
    }
    return p;
}

int err(int code, const char* msg) {
    mm_internal_set_error(msg);
    return code;
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
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return err(MM_ECUDA, "mm_rhs_eval_static: no current CUDA device");
    }
    std::lock_guard<std::mutex> guard(g_lock);
    unsigned char* base = (unsigned char*)scratch_base();
    if (!base) return err(MM_ECUDA, "mm_rhs_eval_static: cudaGetSymbolAddress failed");

    // descriptor of the single simulation (same layout rules as a context: plan.h)
    SimDesc d;
    memset(&d, 0, sizeof(d));
    d.nx = mesh->nx; d.ny = mesh->ny; d.nz = mesh->nz;
    const long long n = (long long)d.nx * d.ny * d.nz;
    if (n > (1LL << 26)) return err(MM_EINVAL, "mm_rhs_eval_static: mesh too large for the static scratch");
    d.ncells = (int)n;
    const int lim = f32 ? 8192 : 4096;
    if (plan_pad_len(d.nx, true) > lim || plan_pad_len(d.ny, false) > lim || plan_pad_len(d.nz, false) > lim)
        return err(MM_EINVAL, f32 ? "mm_rhs_eval_static: padded FFT length too large (max 8192 along each axis in "
                                    "this precision)"
                                  : "mm_rhs_eval_static: padded FFT length too large (max 4096 along each axis in "
                                    "this precision)");
    plan_geometry(d, f32);
    const double un = sqrt(mat->u[0] * mat->u[0] + mat->u[1] * mat->u[1] + mat->u[2] * mat->u[2]);
    if (mat->Ku != 0.0 && !(un > 0)) return err(MM_EINVAL, "mm_rhs_eval_static: anisotropy axis is zero");
    for (int i = 0; i < 3; ++i) { d.u[i] = un > 0 ? mat->u[i] / un : 0.0; d.H[i] = mat->H[i]; }
    d.Ms = mat->Ms; d.A = mat->A; d.D = mat->D; d.Ku = mat->Ku; d.Kc = mat->Kc;
    d.alpha = mat->alpha; d.gamma = mat->gamma;
    d.dx = mesh->dx; d.dy = mesh->dy; d.dz = mesh->dz;
    d.flags = (mat->demag ? F_DEMAG : 0) | (mat->precession ? F_PREC : 0);
    plan_coefficients(d, mat->dmi_kind == MM_DMI_INTERFACIAL);
    d.group_begin = d.group_end = -1;
    d.neb_index = -1;
    d.ms_off = -1;
    d.off = 0;
    d.spec_off = 0;
    d.tens_off = 0;
    const bool demag = mat->demag != 0;
    const size_t vsz = 2 * e;
    PlanItems P;
    plan_items(d, 0, vsz, P);
    const int yzl = plan_uses_yzc(d) ? plan_yzc_list(d, f32) : 0;
    const std::vector<WorkItem>& yzv = P.yzc[yzl];
    const size_t cap = 227 * 1024;
    if (P.smem_x > cap - 4096 || P.smem_xi > cap - 4096 || P.smem_y13 > cap || P.smem_y2 > cap ||
        P.smem_z > cap || P.smem_yzc > cap)
        return err(MM_EINVAL, "mm_rhs_eval_static: FFT tile exceeds shared memory");

    // carve the static array
    Carve cv;
    const size_t o_twd = cv.take((size_t)MM_TW_ENTRIES * 16);
    const size_t o_twf = cv.take((size_t)MM_TW_ENTRIES * 8);
    const size_t o_desc = cv.take(sizeof(SimDesc));
    const size_t o_state = cv.take(sizeof(SimState));
    const size_t o_diag = cv.take(2 * sizeof(unsigned long long));
    const size_t o_xi = cv.take(std::max<size_t>(1, P.x.size()) * sizeof(WorkItem));
    const size_t o_y13 = cv.take(std::max<size_t>(1, P.y13.size()) * sizeof(WorkItem));
    const size_t o_z = cv.take(std::max<size_t>(1, P.z.size()) * sizeof(WorkItem));
    const size_t o_y2 = cv.take(std::max<size_t>(1, P.y2.size()) * sizeof(WorkItem));
    const size_t o_yz = cv.take(std::max<size_t>(1, yzv.size()) * sizeof(WorkItem));
    const long long tens_elems = plan_tens_elems(d);
    const long long spec_elems = demag ? plan_spec_elems(d) : 0;
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
    SCK(up(o_xi, P.x));
    SCK(up(o_y13, P.y13));
    SCK(up(o_z, P.z));
    SCK(up(o_y2, P.y2));
    SCK(up(o_yz, yzv));
    launch_twiddles(s, base + o_twd, base + o_twf, nullptr);   // native FP64 / FP32 transforms here
    upload_gauss_legendre();
    engine_set_attributes();
    SCK(cudaGetLastError());

    if (demag) {
        double* oct = (double*)(base + o_oct);
        void* fftbuf = base + o_fft;
        launch_newell_octant(s, d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, oct);
        const int Tyb = plan_uses_yzc(d) ? d.Ty : 0;   // cluster-pass film: x-y transform, dz planes
        const double scale = Tyb ? 1.0 / ((double)d.Px * d.Py) : 1.0 / ((double)d.Px * d.Py * d.Pz);
        unsigned long long* diag = (unsigned long long*)(base + o_diag);
        SCK(cudaMemsetAsync(base + o_tens, 0, (size_t)tens_elems * e, s));   // padding of a blocked tensor
        for (int c = 0; c < d.ncomp; ++c) {
            launch_newell_place(s, oct, c, d.nx, d.ny, d.nz, d.Px, d.Py, d.Pz, fftbuf);
            for (int ax = 0; ax < (Tyb ? 2 : 3); ++ax)
                launch_fft_axis_f64(s, fftbuf, d.Px, d.Py, d.Pz, ax, base + o_twd);
            launch_newell_extract(s, fftbuf, c, d.Px, d.Py, d.Kx, d.Pyh, Tyb ? d.nz : d.Pzh, scale, base + o_tens,
                                  f32, Tyb, yzc_qp(d.nz), Tyb ? 1 : 0, diag, diag + 1);
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
    L.x = {(const WorkItem*)(base + o_xi), (int)P.x.size()};
    L.y13 = {(const WorkItem*)(base + o_y13), (int)P.y13.size()};
    L.z = {(const WorkItem*)(base + o_z), (int)P.z.size()};
    L.y2 = {(const WorkItem*)(base + o_y2), (int)P.y2.size()};
    if (!yzv.empty()) L.yzc[yzl] = {(const WorkItem*)(base + o_yz), (int)yzv.size()};
    L.smem_x = P.smem_x;
    L.smem_xi = P.smem_xi;
    L.smem_y13 = P.smem_y13;
    L.smem_z = P.smem_z;
    L.smem_y2 = P.smem_y2;
    L.smem_yzc = P.smem_yzc;
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
