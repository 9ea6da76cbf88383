// C ABI of libmm (declared in include/mm.h): contexts, the batch layout,
// work lists, the FP64 tensor precompute, right-hand-side evaluation, graph-
// captured Dormand-Prince attempts, relaxation, energies and NEB chains.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "attempt_small.h"
#include "cayley.h"
#include "engine.cuh"
#include "minimize.h"
#include "potential.h"
#include "mm.h"
#include "plan.h"

using namespace mm;

// the Python binding and other callers lay these out from the header by hand
static_assert(sizeof(mm_mesh) == 40, "mm_mesh layout");
static_assert(sizeof(mm_material) == 120, "mm_material layout");
static_assert(sizeof(mm_status) == 56, "mm_status layout");
static_assert(sizeof(mm_checkpoint) == 64, "mm_checkpoint layout");

namespace {

constexpr double kPi = 3.14159265358979323846;
char g_last_error[512] = "";

struct SimHost {
    mm_mesh mesh;
    mm_material mat;
    std::vector<double> Ms;
    std::vector<double> AD;     // per-cell A then D (2 ncells), empty if uniform
    SimDesc d;
    int geom = -1;
    Tuning tune;                // autotuned / caller-set tiles (0 = rule)
};

struct Geom {
    int nx, ny, nz;
    double dx, dy, dz;
    bool demag = false;
    long long tens_off = -1;    // in the stored tensor (context precision)
    long long oct_off = -1;     // in the FP64 octant table
};

}  // namespace

struct mm_ctx {
    int device = 0;
    int precision = MM_F64;
    size_t esz = 8;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    std::vector<SimHost> sims;
    std::vector<Geom> geoms;
    bool finalized = false;
    long long total_elems = 0, spec_elems = 0, ms_elems = 0, tens_elems = 0, oct_elems = 0, cell_elems = 0;
    void *m = nullptr, *ybuf = nullptr, *k[7] = {}, *errp = nullptr, *spec = nullptr, *Msd = nullptr,
         *tens = nullptr, *twd = nullptr, *twf = nullptr, *twdd = nullptr, *cellp = nullptr;
    bool dd = false;            // FP64 storage with double-float transforms (MM_F64)
    void *sc_in = nullptr, *sc_out = nullptr, *sc_h = nullptr, *heff = nullptr, *tau = nullptr;
    void** kvec_dev = nullptr;
    double* oct = nullptr;
    SimDesc* desc_d = nullptr;
    SimState* state_d = nullptr;
    WorkItem *xi = nullptr, *y13i = nullptr, *zi = nullptr, *y2i = nullptr, *celli = nullptr;
    WorkItem* yzci[kYzcListCount] = {};
    PlanItems plan;
    // per simulation: first item and item count in each list (the yzc list is the
    // one of its plane count and group width, yzcl)
    std::vector<int> xb, xc, y13b, y13c, zb, zc, y2b, y2c, yzcb, yzcc, yzcl, cellb, cellc;
    int *flag_d = nullptr, *status_d = nullptr;
    unsigned long long* diag_d = nullptr;
    cudaGraphExec_t rk_exec = nullptr;
    bool rk_exec_neb = false;
    // steepest-descent minimiser: buffers, per-simulation state, one captured step
    void *sd_H = nullptr, *sd_mprev = nullptr, *sd_g = nullptr;
    SdState* sd_d = nullptr;
    cudaGraphExec_t sd_exec = nullptr;
    long long sd_graph_kernels = 0;
    // fixed-step RK4 (projected or Cayley): one captured step for the last (h, scheme)
    cudaGraphExec_t c4_exec = nullptr;
    double c4_h = 0.0;
    int c4_cay = -1;
    long long c4_graph_kernels = 0;
    // pinned host staging buffer for the host-side state transfers of FP32 contexts
    void* host_stage = nullptr;
    size_t host_stage_bytes = 0;
    // device FP64 staging of FP32 contexts' transfers from and to pinned host buffers
    void* dev_stage = nullptr;
    size_t dev_stage_bytes = 0;
    long long graph_kernels = 0;
    long long launches = 0;
    bool neb = false;
    double tensor_imag_ratio = 0.0;
    // single-launch attempts of small single-plane meshes (attempt_small.cu):
    // MM_ATTEMPT_AUTO or MM_ATTEMPT_PASSES, and the resolved cluster and shared memory
    int attempt_kernel = MM_ATTEMPT_AUTO;
    int small_nc = -1;          // -1 not resolved yet, 0 not eligible
    size_t small_smem = 0;
    // scalar-potential demag (potential.cu): kernel spectrum and work buffers per geometry
    struct PotPlan { PotGeom g; PotBuffers b; };
    std::vector<PotPlan> pot;
};

namespace {

int fail(mm_ctx* C, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (C) C->err = buf;
    snprintf(g_last_error, sizeof(g_last_error), "%s", buf);
    return code;
}

#define CK(x)                                                                                       \
    do {                                                                                            \
        cudaError_t e_ = (x);                                                                       \
        if (e_ != cudaSuccess) return fail(C, MM_ECUDA, "%s: %s", #x, cudaGetErrorString(e_));     \
    } while (0)

int dalloc(mm_ctx* C, void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(C, MM_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    }
    return MM_OK;
}

Launch make_launch(mm_ctx* C, int sim) {
    Launch L;
    L.stream = C->stream;
    L.desc = C->desc_d;
    L.state = C->state_d;
    L.nsims = (int)C->sims.size();
    auto set = [&](ItemSet& is, WorkItem* dev, const std::vector<int>& b, const std::vector<int>& c,
                   const std::vector<WorkItem>& all) {
        if (sim < 0) { is.dev = dev; is.count = (int)all.size(); }
        else { is.dev = dev + b[sim]; is.count = c[sim]; }
    };
    const PlanItems& P = C->plan;
    set(L.x, C->xi, C->xb, C->xc, P.x);
    set(L.y13, C->y13i, C->y13b, C->y13c, P.y13);
    set(L.z, C->zi, C->zb, C->zc, P.z);
    set(L.y2, C->y2i, C->y2b, C->y2c, P.y2);
    set(L.cell, C->celli, C->cellb, C->cellc, P.cell);
    for (int li = 0; li < kYzcListCount; ++li) {
        if (sim < 0) L.yzc[li] = {C->yzci[li], (int)P.yzc[li].size()};
        else if (C->yzcl[sim] == li) L.yzc[li] = {C->yzci[li] + C->yzcb[sim], C->yzcc[sim]};
    }
    L.smem_x = P.smem_x;
    L.smem_xi = P.smem_xi;
    L.smem_y13 = P.smem_y13;
    L.smem_z = P.smem_z;
    L.smem_y2 = P.smem_y2;
    L.smem_yzc = P.smem_yzc;
    // launch-wide CTA widths: the tuned value when every simulation has the same one
    L.x_threads = C->sims.empty() ? 0 : C->sims[0].tune.x_threads;
    L.col_threads = C->sims.empty() ? 0 : C->sims[0].tune.col_threads;
    for (const SimHost& s : C->sims) {
        if (s.tune.x_threads != L.x_threads) L.x_threads = 0;
        if (s.tune.col_threads != L.col_threads) L.col_threads = 0;
    }
    L.tensor = C->tens;
    L.Ms = C->Msd;
    L.cellp = C->cellp;
    for (const SimHost& s : C->sims) L.ext = L.ext || (s.d.flags & F_EXT) != 0;
    L.tw = C->precision == MM_F32 ? C->twf : (C->dd ? C->twdd : C->twd);
    L.dd = C->dd;
    L.spec = C->spec;
    L.launches = &C->launches;
    return L;
}

// Term flags and coefficients of one simulation from its parameters.
void replan(SimHost& s) {
    plan_coefficients(s.d, s.mat.dmi_kind == MM_DMI_INTERFACIAL);
    bool a_any = false, d_any = false;
    const size_t n = s.AD.size() / 2;
    for (size_t i = 0; i < n; ++i) {
        a_any = a_any || s.AD[i] != 0.0;
        d_any = d_any || s.AD[n + i] != 0.0;
    }
    plan_extended(s.d, !s.AD.empty(), a_any, d_any);
}

bool batch_ext(const mm_ctx* C) {
    for (const SimHost& s : C->sims)
        if (s.d.flags & F_EXT) return true;
    return false;
}

// Captured graphs bake in the x-inverse variant; drop them when it changes.
void drop_graphs(mm_ctx* C) {
    if (C->rk_exec) { cudaGraphExecDestroy(C->rk_exec); C->rk_exec = nullptr; }
    if (C->sd_exec) { cudaGraphExecDestroy(C->sd_exec); C->sd_exec = nullptr; }
    if (C->c4_exec) { cudaGraphExecDestroy(C->c4_exec); C->c4_exec = nullptr; }
}

int check_ready(mm_ctx* C) {
    if (!C) return MM_EINVAL;
    if (!C->finalized) return fail(C, MM_EINVAL, "call mm_precompute_demag first");
    return MM_OK;
}

// Every global index a work item can touch, checked on the host before any launch.
// Kernels index inside the per-simulation blocks checked here (state [3][N],
// spectrum [3][nz][NBx][Py][Ty], tensor [ncomp][Pzh][Pyh][Kx]) from item
// coordinates checked here.
int validate_items(mm_ctx* C) {
    const PlanItems& P = C->plan;
    const size_t vsz = 2 * C->esz;
    for (const SimHost& s : C->sims) {
        const SimDesc& d = s.d;
        if (d.off < 0 || d.off + 3LL * d.ncells > C->total_elems) return fail(C, MM_EBOUNDS, "state block");
        if (d.flags & F_DEMAG) {
            if (d.spec_off < 0 || d.spec_off + plan_spec_elems(d) > C->spec_elems)
                return fail(C, MM_EBOUNDS, "spectrum block");
            if (d.tens_off < 0 || d.tens_off + plan_tens_elems(d) > C->tens_elems)
                return fail(C, MM_EBOUNDS, "tensor block");
            if ((d.NBx << d.lTy) < d.Kx || d.Ty != (1 << d.lTy)) return fail(C, MM_EBOUNDS, "kx blocks");
        }
        if (d.ms_off >= 0 && d.ms_off + d.ncells > C->ms_elems) return fail(C, MM_EBOUNDS, "Ms array");
        if ((d.eflags & E_CELL) && (d.cell_off < 0 || d.cell_off + 2LL * d.ncells > C->cell_elems))
            return fail(C, MM_EBOUNDS, "per-cell A and D block");
    }
    for (const WorkItem& w : P.x) {
        const SimDesc& d = C->sims[w.sim].d;
        if (w.a < 0 || w.b < 1 || w.a + w.b > d.ny * d.nz) return fail(C, MM_EBOUNDS, "x item rows");
        if (2 * 3ULL * w.b * padded_len(d.Kx) * vsz > P.smem_x) return fail(C, MM_EBOUNDS, "x item smem");
        if ((d.flags & F_XSTAGE) &&
            xinv_stage_offset(3 * w.b, padded_len(d.Kx), vsz) + xinv_stage_bytes(w.b, d.nx, C->esz) > P.smem_xi)
            return fail(C, MM_EBOUNDS, "x-inverse staged rows smem");
        if ((w.a % d.ny) + w.b > d.ny) return fail(C, MM_EBOUNDS, "x item crosses a plane");
        if (plan_spec_elems(d) >= (1LL << 31) || 3LL * d.ncells >= (1LL << 31))
            return fail(C, MM_EINVAL, "simulation too large for 32-bit per-simulation offsets");
    }
    for (const WorkItem& w : P.cell) {
        const SimDesc& d = C->sims[w.sim].d;
        if (w.a < 0 || w.b < 1 || w.a + w.b > d.ny * d.nz || (w.a % d.ny) + w.b > d.ny)
            return fail(C, MM_EBOUNDS, "cell tile rows");
    }
    for (const WorkItem& w : P.y13) {
        const SimDesc& d = C->sims[w.sim].d;
        if (w.a < 0 || w.a >= d.nz || w.b < 0 || w.b >= d.NBx || w.c < 0 || w.c > 2)
            return fail(C, MM_EBOUNDS, "y item range");
        if ((size_t)d.Py * d.Ty * vsz > P.smem_y13) return fail(C, MM_EBOUNDS, "y item smem");
    }
    for (const WorkItem& w : P.y2) {
        const SimDesc& d = C->sims[w.sim].d;
        if (w.a != 0 || d.nz != 1 || w.b < 0 || w.b >= d.NBx) return fail(C, MM_EBOUNDS, "y2 item range");
        if (3ULL * d.Py * d.Ty * vsz > P.smem_y2) return fail(C, MM_EBOUNDS, "y2 item smem");
    }
    for (const WorkItem& w : P.z) {
        const SimDesc& d = C->sims[w.sim].d;
        if (w.a < 0 || w.a >= d.Py || w.b < 0 || w.b >= d.NBx) return fail(C, MM_EBOUNDS, "z item range");
        if (3ULL * d.Pz * d.Ty * vsz > P.smem_z) return fail(C, MM_EBOUNDS, "z item smem");
    }
    for (int li = 0; li < kYzcListCount; ++li) {
        const int nz = plan_yzc_nz(li);
        for (const WorkItem& w : P.yzc[li]) {
            const SimDesc& d = C->sims[w.sim].d;
            if (d.nz != nz || d.Py < 2 || w.b < 0 || w.b >= d.NBx || d.Pz != plan_pad_len(nz, false) ||
                plan_yzc_list(d, C->precision == MM_F32) != li)
                return fail(C, MM_EBOUNDS, "yz item range");
            if (3ULL * d.Py * d.Ty * vsz > P.smem_yzc) return fail(C, MM_EBOUNDS, "yz item smem");
        }
    }
    const size_t cap = 227 * 1024;
    if (P.smem_x > cap - 4096 || P.smem_xi > cap - 4096 || P.smem_y13 > cap || P.smem_y2 > cap || P.smem_z > cap ||
        P.smem_yzc > cap)
        return fail(C, MM_EINVAL, "a padded FFT length needs more shared memory than one CTA has");
    return MM_OK;
}

int upload_descs(mm_ctx* C) {
    C->small_nc = -1;           // term flags may have changed: resolve the attempt path again
    std::vector<SimDesc> h(C->sims.size());
    for (size_t i = 0; i < C->sims.size(); ++i) h[i] = C->sims[i].d;
    CK(cudaMemcpyAsync(C->desc_d, h.data(), h.size() * sizeof(SimDesc), cudaMemcpyHostToDevice, C->stream));
    CK(cudaStreamSynchronize(C->stream));
    return MM_OK;
}

int read_states(mm_ctx* C, std::vector<SimState>& st) {
    st.resize(C->sims.size());
    CK(cudaMemcpyAsync(st.data(), C->state_d, st.size() * sizeof(SimState), cudaMemcpyDeviceToHost, C->stream));
    CK(cudaStreamSynchronize(C->stream));
    return MM_OK;
}

int write_states(mm_ctx* C, const std::vector<SimState>& st) {
    CK(cudaMemcpyAsync(C->state_d, st.data(), st.size() * sizeof(SimState), cudaMemcpyHostToDevice, C->stream));
    CK(cudaStreamSynchronize(C->stream));
    return MM_OK;
}

// FP64 octant table and stored spectrum of one geometry
int precompute_geometry(mm_ctx* C, Geom& g, const SimDesc& d) {
    launch_newell_octant(C->stream, g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, C->oct + g.oct_off);
    C->launches += 1;
    CK(cudaGetLastError());
    if (!g.demag) return MM_OK;
    void* buf = nullptr;
    const size_t bytes = (size_t)d.Px * d.Py * d.Pz * 16;
    int rc = dalloc(C, &buf, bytes);
    if (rc) return rc;
    // films of the cluster pass convolve along z directly: their tensor is transformed
    // along x and y only, one value per dz = 0..nz-1 (plan_tens_elems)
    const bool blocked = plan_uses_yzc(d);
    const double scale = blocked ? 1.0 / ((double)d.Px * d.Py) : 1.0 / ((double)d.Px * d.Py * d.Pz);
    // the spectrum of an even/odd real tensor is real (along x, y only: xz, yz are
    // imaginary): compare the largest discarded part with the largest kept part
    CK(cudaMemsetAsync(C->diag_d, 0, 2 * sizeof(unsigned long long), C->stream));
    for (int c = 0; c < d.ncomp; ++c) {
        launch_newell_place(C->stream, C->oct + g.oct_off, c, g.nx, g.ny, g.nz, d.Px, d.Py, d.Pz, buf);
        for (int ax = 0; ax < (blocked ? 2 : 3); ++ax)
            launch_fft_axis_f64(C->stream, buf, d.Px, d.Py, d.Pz, ax, C->twd);
        char* out = (char*)C->tens + (size_t)g.tens_off * C->esz;
        launch_newell_extract(C->stream, buf, c, d.Px, d.Py, d.Kx, d.Pyh, blocked ? d.nz : d.Pzh, scale, out,
                              C->precision == MM_F32 ? 1 : (C->dd ? 2 : 0), blocked ? d.Ty : 0, yzc_qp(d.nz),
                              blocked ? 1 : 0,
                              C->diag_d, C->diag_d + 1);
        C->launches += blocked ? 4 : 5;
        CK(cudaGetLastError());
    }
    unsigned long long hb[2];
    CK(cudaMemcpyAsync(hb, C->diag_d, sizeof(hb), cudaMemcpyDeviceToHost, C->stream));
    CK(cudaStreamSynchronize(C->stream));
    double im, re;
    memcpy(&im, &hb[0], 8);
    memcpy(&re, &hb[1], 8);
    const double worst = re > 0 ? im / re : 0.0;
    cudaFree(buf);
    C->tensor_imag_ratio = std::max(C->tensor_imag_ratio, worst);
    if (!(worst < 1e-9)) return fail(C, MM_ECUDA, "tensor spectrum not real (|Im|/|Re| = %g)", worst);
    return MM_OK;
}

template <typename T>
void to_prec(const double* src, T* dst, size_t n) {
    for (size_t i = 0; i < n; ++i) dst[i] = (T)src[i];
}

// Element-wise conversion of a large host array on several host threads.
template <typename A, typename B>
void convert_host(const A* src, B* dst, long long n) {
    const unsigned hc = std::thread::hardware_concurrency();
    const int nt = n < (1LL << 18) ? 1 : (int)std::min(8u, std::max(1u, hc));
    if (nt == 1) {
        for (long long i = 0; i < n; ++i) dst[i] = (B)src[i];
        return;
    }
    std::vector<std::thread> th;
    const long long chunk = (n + nt - 1) / nt;
    for (int t = 0; t < nt; ++t) {
        const long long lo = t * chunk, hi = std::min(n, lo + chunk);
        th.emplace_back([=] { for (long long i = lo; i < hi; ++i) dst[i] = (B)src[i]; });
    }
    for (auto& x : th) x.join();
}

// FP64 <-> FP32 conversion of a state on the device (transfers of FP32 contexts
// from and to pinned host buffers: the FP64 values cross the link by DMA and the
// rounding to FP32 is the same (T)x as on the host)
template <typename A, typename B>
__global__ void k_convert(const A* __restrict__ src, B* __restrict__ dst, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = (B)src[i];
}

// Whether a host pointer is page-locked (cudaMallocHost or registered): then the
// FP64 values go by DMA and are converted on the device.
bool host_pinned(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

int ensure_dev_stage(mm_ctx* C, size_t bytes) {
    if (C->dev_stage_bytes >= bytes) return MM_OK;
    if (C->dev_stage) cudaFree(C->dev_stage);
    C->dev_stage = nullptr;
    C->dev_stage_bytes = 0;
    int rc = dalloc(C, &C->dev_stage, bytes);
    if (rc) return rc;
    C->dev_stage_bytes = bytes;
    return MM_OK;
}

static unsigned convert_blocks(long long n) { return (unsigned)std::min<long long>((n + 255) / 256, 4096); }

// The pinned staging buffer, grown to at least `bytes` (reused by every host transfer).
int ensure_host_stage(mm_ctx* C, size_t bytes) {
    if (C->host_stage_bytes >= bytes) return MM_OK;
    if (C->host_stage) cudaFreeHost(C->host_stage);
    C->host_stage = nullptr;
    C->host_stage_bytes = 0;
    const cudaError_t e = cudaMallocHost(&C->host_stage, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(C, MM_ENOMEM, "cudaMallocHost(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    }
    C->host_stage_bytes = bytes;
    return MM_OK;
}

int ensure_scratch(mm_ctx* C) {
    if (C->sc_in) return MM_OK;
    const size_t b = (size_t)C->total_elems * C->esz;
    int rc;
    if ((rc = dalloc(C, &C->sc_in, b))) return rc;
    if ((rc = dalloc(C, &C->sc_out, b))) return rc;
    if ((rc = dalloc(C, &C->sc_h, b))) return rc;
    return MM_OK;
}

int build_graph(mm_ctx* C) {
    if (C->rk_exec && C->rk_exec_neb == C->neb) return MM_OK;
    if (C->rk_exec) { cudaGraphExecDestroy(C->rk_exec); C->rk_exec = nullptr; }
    Launch L = make_launch(C, -1);
    RkBuffers B;
    B.m = C->m;
    B.ybuf = C->ybuf;
    B.kvec_dev = C->kvec_dev;
    for (int j = 0; j < 7; ++j) B.kvec[j] = C->k[j];
    B.errp = C->errp;
    B.heff = C->heff;
    B.tau = C->tau;
    const long long before = C->launches;
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(C->stream, cudaStreamCaptureModeThreadLocal));
    if (C->precision == MM_F32) {
        if (C->neb) engine_neb_attempt<float>(L, B); else engine_attempt<float>(L, B);
    } else {
        if (C->neb) engine_neb_attempt<double>(L, B); else engine_attempt<double>(L, B);
    }
    cudaError_t e = cudaStreamEndCapture(C->stream, &g);
    if (e != cudaSuccess) return fail(C, MM_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&C->rk_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(C, MM_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    C->graph_kernels = C->launches - before;
    C->launches = before;
    C->rk_exec_neb = C->neb;
    return MM_OK;
}

// Whether every simulation can run its attempts in one launch (attempt_small.cu),
// and on which cluster: the largest of 16, 8, 4, 2, 1 CTAs a simulation that the
// device co-schedules.  When the whole batch fits on the SMs at one CTA each, the
// dynamic shared memory is raised so that no two CTAs share an SM (the FP64
// epilogue is bound by each SM's FP64 rate).
void small_resolve(mm_ctx* C) {
    C->small_nc = 0;
    if (C->attempt_kernel == MM_ATTEMPT_PASSES || C->neb || C->sims.empty()) return;
    for (const SimHost& s : C->sims)
        if (!small_eligible(s.d)) return;
    const int kind = C->precision == MM_F32 ? 0 : (C->dd ? 2 : 1);
    const size_t ssz = C->esz, csz = C->precision == MM_F32 ? 4 : 8;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, C->device);
    const int top = C->attempt_kernel >= 2 ? C->attempt_kernel : kSmallMaxCluster;
    for (int nc = top; nc >= 1; nc >>= 1) {
        size_t smem = 0;
        for (const SimHost& s : C->sims) smem = std::max(smem, small_smem_bytes(s.d, nc, ssz, csz));
        if ((long long)C->sims.size() * nc <= sms) smem = std::max<size_t>(smem, 116 * 1024);
        if (small_cluster_fits(kind, smem, nc)) {
            C->small_nc = nc;
            C->small_smem = smem;
            return;
        }
    }
}

int launch_attempts(mm_ctx* C, long long n) {
    if (C->small_nc < 0) small_resolve(C);
    if (C->small_nc > 0 && !C->neb) {
        SmallLaunch S;
        S.stream = C->stream;
        S.desc = C->desc_d;
        S.state = C->state_d;
        S.nsims = (int)C->sims.size();
        S.m = C->m;
        S.tensor = C->tens;
        S.Ms = C->Msd;
        S.tw = C->precision == MM_F32 ? C->twf : (C->dd ? C->twdd : C->twd);
        S.kind = C->precision == MM_F32 ? 0 : (C->dd ? 2 : 1);
        S.cluster = C->small_nc;
        S.smem = C->small_smem;
        // at most 1024 attempts a launch, so no single kernel runs for long
        for (long long done = 0; done < n;) {
            const long long chunk = std::min<long long>(n - done, 1024);
            S.n_attempts = (int)chunk;
            CK(small_attempts(S));
            C->launches += 1;
            done += chunk;
        }
        return MM_OK;
    }
    int rc = build_graph(C);
    if (rc) return rc;
    for (long long i = 0; i < n; ++i) {
        CK(cudaGraphLaunch(C->rk_exec, C->stream));
        C->launches += C->graph_kernels;
    }
    return MM_OK;
}

// Buffers of the minimiser and one captured step (the step reads everything it
// needs from device memory, so the graph stays valid for every call).
int sd_prepare(mm_ctx* C) {
    int rc;
    const size_t sb = (size_t)C->total_elems * C->esz;
    if (!C->sd_H) {
        if ((rc = ensure_scratch(C))) return rc;
        if ((rc = dalloc(C, &C->sd_H, sb))) return rc;
        if ((rc = dalloc(C, &C->sd_mprev, sb))) return rc;
        if ((rc = dalloc(C, &C->sd_g, sb))) return rc;
        if ((rc = dalloc(C, (void**)&C->sd_d, C->sims.size() * sizeof(SdState)))) return rc;
    }
    if (C->sd_exec) return MM_OK;
    Launch L = make_launch(C, -1);
    SdBuffers B;
    B.m = C->m;
    B.H = C->sd_H;
    B.dmdt = C->sc_out;
    B.mprev = C->sd_mprev;
    B.gprev = C->sd_g;
    B.sd = C->sd_d;
    const long long before = C->launches;
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(C->stream, cudaStreamCaptureModeThreadLocal));
    if (C->precision == MM_F32) sd_step<float>(L, B); else sd_step<double>(L, B);
    cudaError_t e = cudaStreamEndCapture(C->stream, &g);
    if (e != cudaSuccess) return fail(C, MM_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&C->sd_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(C, MM_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    C->sd_graph_kernels = C->launches - before;
    C->launches = before;
    return MM_OK;
}

// One captured RK4 step; the step size is a kernel argument, so a call with
// another h or scheme captures again.  Stage slopes live in the RK45 stage
// buffers, the stage state in its stage-state buffer (neither carries state
// from one RK45 attempt to the next).
int c4_prepare(mm_ctx* C, double h, int cay) {
    int rc;
    if ((rc = ensure_scratch(C))) return rc;
    if (C->c4_exec && C->c4_h == h && C->c4_cay == cay) return MM_OK;
    if (C->c4_exec) { cudaGraphExecDestroy(C->c4_exec); C->c4_exec = nullptr; }
    Launch L = make_launch(C, -1);
    Rk4Buffers B;
    B.m = C->m;
    B.ys = C->ybuf;
    B.H = C->sc_h;
    B.dmdt = C->sc_out;
    for (int j = 0; j < 4; ++j) B.k[j] = C->k[j];
    const long long before = C->launches;
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(C->stream, cudaStreamCaptureModeThreadLocal));
    if (C->precision == MM_F32) rk4_step<float>(L, B, h, cay != 0); else rk4_step<double>(L, B, h, cay != 0);
    cudaError_t e = cudaStreamEndCapture(C->stream, &g);
    if (e != cudaSuccess) return fail(C, MM_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&C->c4_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(C, MM_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    C->c4_graph_kernels = C->launches - before;
    C->launches = before;
    C->c4_h = h;
    C->c4_cay = cay;
    return MM_OK;
}

int first_error(mm_ctx* C, const std::vector<SimState>& st) {
    for (size_t i = 0; i < st.size(); ++i) {
        if (st[i].status < 0) {
            const int s = st[i].status;
            return fail(C, s, "simulation %zu: %s", i,
                        s == MM_ENAN ? "non-finite error norm"
                        : s == MM_ESTEP ? "step size underflow"
                        : s == MM_ETIMEOUT ? "a staged copy into shared memory did not complete (bounded wait)"
                                           : "error");
        }
    }
    return MM_OK;
}

}  // namespace

extern "C" {

const char* mm_last_error(const mm_ctx* C) { return C ? C->err.c_str() : g_last_error; }

int mm_create(mm_ctx** out, int device, int precision, void* cuda_stream) {
    if (!out) return fail(nullptr, MM_EINVAL, "out is NULL");
    *out = nullptr;
    if (precision != MM_F64 && precision != MM_F32 && precision != MM_F64_NATIVE)
        return fail(nullptr, MM_EINVAL, "precision must be MM_F64, MM_F32 or MM_F64_NATIVE");
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) {
        cudaGetLastError();
        return fail(nullptr, MM_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
    }
    if (device < 0 || device >= n) return fail(nullptr, MM_EINVAL, "device %d out of range", device);
    mm_ctx* C = new mm_ctx;
    C->device = device;
    C->precision = precision == MM_F32 ? MM_F32 : MM_F64;
    C->dd = precision == MM_F64;
    C->esz = precision == MM_F32 ? 4 : 8;
    e = cudaSetDevice(device);
    if (e != cudaSuccess) { delete C; return fail(nullptr, MM_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e)); }
    if (cuda_stream) C->stream = (cudaStream_t)cuda_stream;
    else {
        e = cudaStreamCreateWithFlags(&C->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete C; return fail(nullptr, MM_ECUDA, "stream: %s", cudaGetErrorString(e)); }
        C->own_stream = true;
    }
    *out = C;
    return MM_OK;
}

int mm_destroy(mm_ctx* C) {
    if (!C) return MM_EINVAL;
    cudaSetDevice(C->device);
    if (C->stream) cudaStreamSynchronize(C->stream);
    if (C->rk_exec) cudaGraphExecDestroy(C->rk_exec);
    if (C->sd_exec) cudaGraphExecDestroy(C->sd_exec);
    if (C->c4_exec) cudaGraphExecDestroy(C->c4_exec);
    void* ptrs[] = {C->m, C->ybuf, C->errp, C->spec, C->Msd, C->cellp, C->tens, C->twd, C->twf, C->twdd, C->sc_in,
                    C->sc_out,
                    C->sc_h, C->heff, C->tau, C->kvec_dev, C->oct, C->desc_d, C->state_d, C->xi, C->y13i,
                    C->zi, C->y2i, C->celli, C->flag_d, C->status_d, C->diag_d, C->sd_H, C->sd_mprev, C->sd_g,
                    C->sd_d};
    for (void* p : ptrs) if (p) cudaFree(p);
    for (auto& pp : C->pot) {
        void* pb[] = {pp.b.Shat, pp.b.Mhat, pp.b.U, pp.b.u};
        for (void* p : pb) if (p) cudaFree(p);
    }
    if (C->host_stage) cudaFreeHost(C->host_stage);
    if (C->dev_stage) cudaFree(C->dev_stage);
    for (int j = 0; j < 7; ++j) if (C->k[j]) cudaFree(C->k[j]);
    for (int li = 0; li < kYzcListCount; ++li) if (C->yzci[li]) cudaFree(C->yzci[li]);
    if (C->own_stream) cudaStreamDestroy(C->stream);
    delete C;
    return MM_OK;
}

int mm_add_sim(mm_ctx* C, const mm_mesh* mesh, const mm_material* mat, const double* Ms_cells, int* sim_id) {
    if (!C || !mesh || !mat) return fail(C, MM_EINVAL, "NULL argument");
    if (C->finalized) return fail(C, MM_EINVAL, "mm_add_sim after mm_precompute_demag");
    if (mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1) return fail(C, MM_EINVAL, "mesh dims must be >= 1");
    if (!(mesh->dx > 0 && mesh->dy > 0 && mesh->dz > 0)) return fail(C, MM_EINVAL, "cell sizes must be > 0");
    const long long ncells = (long long)mesh->nx * mesh->ny * mesh->nz;
    if (ncells > (1LL << 30)) return fail(C, MM_EINVAL, "mesh too large");
    if (!(mat->Ms >= 0) || !(mat->alpha >= 0) || !(mat->gamma > 0))
        return fail(C, MM_EINVAL, "Ms, alpha must be >= 0 and gamma > 0");
    SimHost s;
    s.mesh = *mesh;
    s.mat = *mat;
    SimDesc& d = s.d;
    memset(&d, 0, sizeof(d));
    d.nx = mesh->nx; d.ny = mesh->ny; d.nz = mesh->nz;
    d.ncells = (int)ncells;
    // one x row (two padded buffers of three components) and one column tile must fit a CTA's shared memory
    const int lim = C->precision == MM_F32 ? 8192 : 4096;
    if (plan_pad_len(d.nx, true) > lim || plan_pad_len(d.ny, false) > lim || plan_pad_len(d.nz, false) > lim)
        return fail(C, MM_EINVAL, "padded FFT length too large (max %d along each axis in this precision)", lim);
    plan_geometry(d, C->precision == MM_F32);
    double un = std::sqrt(mat->u[0] * mat->u[0] + mat->u[1] * mat->u[1] + mat->u[2] * mat->u[2]);
    if (mat->Ku != 0.0 && !(un > 0)) return fail(C, MM_EINVAL, "anisotropy axis is zero");
    for (int i = 0; i < 3; ++i) d.u[i] = un > 0 ? mat->u[i] / un : 0.0;
    d.Ms = mat->Ms; d.A = mat->A; d.D = mat->D; d.Ku = mat->Ku; d.Kc = mat->Kc;
    for (int i = 0; i < 3; ++i) d.H[i] = mat->H[i];
    d.alpha = mat->alpha; d.gamma = mat->gamma;
    d.dx = mesh->dx; d.dy = mesh->dy; d.dz = mesh->dz;
    d.flags = (mat->demag ? F_DEMAG : 0) | (mat->precession ? F_PREC : 0);
    if (mat->dmi_kind < MM_DMI_NONE || mat->dmi_kind > MM_DMI_D2D) return fail(C, MM_EINVAL, "unsupported DMI kind");
    d.dmi_kind = mat->dmi_kind;
    d.cell_off = -1;
    d.p[2] = 1.0;
    replan(s);
    d.group_begin = d.group_end = -1;
    d.neb_index = -1;
    d.ms_off = -1;
    if (Ms_cells) {
        s.Ms.assign(Ms_cells, Ms_cells + ncells);
        for (double v : s.Ms) if (!(v >= 0)) return fail(C, MM_EINVAL, "per-cell Ms must be >= 0");
        d.flags |= F_MSARR;
    }
    C->sims.push_back(std::move(s));
    if (sim_id) *sim_id = (int)C->sims.size() - 1;
    return MM_OK;
}

int mm_num_sims(const mm_ctx* C) { return C ? (int)C->sims.size() : MM_EINVAL; }

namespace {

Tuning from_abi(const mm_tuning& t) {
    Tuning u;
    u.Ty = t.Ty; u.Rx = t.Rx; u.x_threads = t.x_threads; u.col_threads = t.col_threads; u.col_group = t.col_group;
    u.col_occ = t.col_occ;
    u.x_stage = t.x_stage;
    return u;
}

// Plan sim s with tuning t (before finalisation); MM_EINVAL if its tiles do not fit.
int apply_tuning(mm_ctx* C, SimHost& s, const Tuning& t) {
    const bool f32 = C->precision == MM_F32;
    if (t.Ty < 0 || t.Rx < 0 || t.x_threads < 0 || t.col_threads < 0 || t.col_group < 0 || t.col_group > 2 ||
        (t.col_occ != 0 && t.col_occ != 2 && t.col_occ != 3 && t.col_occ != 4) || t.x_stage < 0 || t.x_stage > 2)
        return fail(C, MM_EINVAL, "mm_set_tuning: negative or unknown value");
    if (t.Ty > 32 || (t.Ty & (t.Ty - 1))) return fail(C, MM_EINVAL, "mm_set_tuning: Ty must be a power of two <= 32");
    SimDesc d = s.d;
    plan_geometry(d, f32, t);
    if (!plan_tuning_valid(d, 2 * C->esz, t, f32 ? 1024 : 512))
        return fail(C, MM_EINVAL, "mm_set_tuning: tiles exceed the kernels' limits (Ty %d, Rx %d, threads %d / %d)",
                    d.Ty, d.Rx, t.x_threads, t.col_threads);
    s.d = d;
    s.tune = t;
    return MM_OK;
}

// The tuning of s with every rule value filled in.
mm_tuning resolved_tuning(const mm_ctx* C, const SimHost& s) {
    const bool f32 = C->precision == MM_F32;
    const int maxth = f32 ? 1024 : 512;
    PlanItems P;
    SimDesc e = s.d;
    e.flags |= F_DEMAG;
    plan_items(e, 0, 2 * C->esz, P);
    mm_tuning r;
    r.Ty = s.d.Ty;
    r.Rx = s.d.Rx;
    r.x_threads = s.tune.x_threads ? s.tune.x_threads : plan_wide_threads(P.smem_x, maxth);
    const size_t sc = std::max(P.smem_y13, std::max(P.smem_z, P.smem_y2));
    r.col_threads = s.tune.col_threads ? s.tune.col_threads : (sc ? plan_wide_threads(sc, maxth) : 0);
    r.col_group = plan_uses_yzc(s.d) ? (plan_yzc_wide(plan_yzc_list(s.d, f32)) ? 2 : 1) : 0;
    r.col_occ = plan_uses_yzc(s.d) ? s.d.yzcocc : 0;
    r.x_stage = (s.d.flags & F_XSTAGE) ? 1 : 0;
    return r;
}

bool same_mesh(const mm_mesh& a, const mm_mesh& b) {
    return a.nx == b.nx && a.ny == b.ny && a.nz == b.nz && a.dx == b.dx && a.dy == b.dy && a.dz == b.dz;
}

// Tuning t for the simulations of the tuned mesh, and t's launch-wide CTA widths
// (which act on the whole batch) with its own tiles for any other simulation.
Tuning tuning_for(const SimHost& o, const mm_mesh& tuned, const Tuning& t) {
    if (same_mesh(o.mesh, tuned)) return t;
    Tuning u = o.tune;
    u.x_threads = t.x_threads;
    u.col_threads = t.col_threads;
    return u;
}

// Milliseconds per RK45 attempt of a copy of C's whole batch with tuning t on the
// simulations of `tuned`'s mesh, in a scratch context on C's device (two untimed
// attempts, then `reps` timed): the batch as it will run, so a mesh is tuned for
// the launches it shares with the other meshes.
int time_tuning(mm_ctx* C, const mm_mesh& tuned, const Tuning& t, int reps, double* ms) {
    mm_ctx* T = nullptr;
    int rc = mm_create(&T, C->device, C->precision == MM_F32 ? MM_F32 : (C->dd ? MM_F64 : MM_F64_NATIVE), nullptr);
    if (rc) return fail(C, rc, "mm_autotune: scratch context: %s", g_last_error);
    for (const SimHost& o : C->sims) {
        SimHost h = o;
        h.d.group_begin = h.d.group_end = -1;
        h.d.neb_index = -1;
        T->sims.push_back(h);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto done = [&](int code) -> int {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (code && code != MM_OK) { std::string m = T->err; mm_destroy(T); return fail(C, code, "mm_autotune: %s", m.c_str()); }
        mm_destroy(T);
        return MM_OK;
    };
    for (SimHost& h : T->sims)
        if ((rc = apply_tuning(T, h, tuning_for(h, tuned, t)))) return done(rc);
    if ((rc = mm_precompute_demag(T))) return done(rc);
    for (size_t j = 0; j < T->sims.size(); ++j) {
        const long long N = T->sims[j].d.ncells;
        std::vector<double> m(3 * N);
        for (long long i = 0; i < N; ++i) {      // a smooth unit-vector texture
            const double a = 0.37 * (double)(i % 97), b = 0.11 * (double)(i % 89);
            m[i] = std::cos(a) * std::sin(b + 0.3);
            m[N + i] = std::sin(a) * std::sin(b + 0.3);
            m[2 * N + i] = std::cos(b + 0.3);
        }
        if ((rc = mm_set_m(T, (int)j, m.data(), MM_HOST))) return done(rc);
    }
    if ((rc = mm_rk45_setup(T, 1e-5, 0.0, 0.0))) return done(rc);
    if ((rc = launch_attempts(T, 2))) return done(rc);
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return done(MM_ECUDA);
    cudaEventRecord(e0, T->stream);
    if ((rc = launch_attempts(T, reps))) return done(rc);
    cudaEventRecord(e1, T->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) return done(MM_ECUDA);
    float t_ms = 0.f;
    cudaEventElapsedTime(&t_ms, e0, e1);
    *ms = (double)t_ms / reps;
    return done(MM_OK);
}

}  // namespace

int mm_set_tuning(mm_ctx* C, int sim, const mm_tuning* t) {
    if (!C || !t) return fail(C, MM_EINVAL, "NULL argument");
    if (C->finalized) return fail(C, MM_EINVAL, "mm_set_tuning after mm_precompute_demag");
    if (sim < -1 || sim >= (int)C->sims.size()) return fail(C, MM_EINVAL, "bad sim id");
    for (int i = (sim < 0 ? 0 : sim); i < (sim < 0 ? (int)C->sims.size() : sim + 1); ++i) {
        const int rc = apply_tuning(C, C->sims[i], from_abi(*t));
        if (rc) return rc;
    }
    return MM_OK;
}

int mm_get_tuning(const mm_ctx* C, int sim, mm_tuning* out) {
    if (!C || !out || sim < 0 || sim >= (int)C->sims.size()) return MM_EINVAL;
    *out = resolved_tuning(C, C->sims[sim]);
    return MM_OK;
}

int mm_autotune(mm_ctx* C, int sim, int reps, mm_tuning* best_out, double* best_ms, double* rule_ms) {
    if (!C) return MM_EINVAL;
    if (C->finalized) return fail(C, MM_EINVAL, "mm_autotune after mm_precompute_demag");
    if (sim < 0 || sim >= (int)C->sims.size() || reps < 1) return fail(C, MM_EINVAL, "bad arguments");
    const bool f32 = C->precision == MM_F32;
    const SimHost& s = C->sims[sim];
    const mm_mesh mesh = s.mesh;
    SimDesc r = s.d;
    plan_geometry(r, f32);                       // the rule
    Tuning best;
    best.Ty = r.Ty;
    best.Rx = r.Rx;
    best.x_threads = s.tune.x_threads;           // launch-wide: as the batch has them
    best.col_threads = s.tune.col_threads;
    best.col_group = (f32 && plan_uses_yzc(r)) ? (plan_yzc_wide(plan_yzc_list(r, f32)) ? 2 : 1) : 0;
    double tbest = 0.0, trule = 0.0;
    bool first = true;
    for (int phase = 0; phase < 3; ++phase) {
        const std::vector<Tuning> cand = plan_tuning_candidates(r, f32, phase, best);
        const Tuning fixed = best;
        for (size_t i = 0; i < cand.size(); ++i) {
            if (i == 0 && !first) continue;      // the phase's starting point was timed already
            double ms = 0.0;
            const int rc = time_tuning(C, mesh, cand[i], reps, &ms);
            if (rc) return rc;
            if (first) { trule = ms; tbest = ms; best = cand[i]; first = false; continue; }
            if (ms < tbest) { tbest = ms; best = cand[i]; }
        }
        (void)fixed;
    }
    for (SimHost& o : C->sims) {
        const int rc = apply_tuning(C, o, tuning_for(o, mesh, best));
        if (rc) return rc;
    }
    if (best_out) {
        best_out->Ty = best.Ty; best_out->Rx = best.Rx; best_out->x_threads = best.x_threads;
        best_out->col_threads = best.col_threads; best_out->col_group = best.col_group;
        best_out->col_occ = best.col_occ;
        best_out->x_stage = best.x_stage;
    }
    if (best_ms) *best_ms = tbest;
    if (rule_ms) *rule_ms = trule;
    return MM_OK;
}

int mm_batch_layout(const mm_ctx* C, long long* offsets, long long* total) {
    if (!C) return MM_EINVAL;
    long long off = 0;
    for (size_t i = 0; i < C->sims.size(); ++i) {
        if (offsets) offsets[i] = off;
        off += 3LL * C->sims[i].d.ncells;
    }
    if (total) *total = off;
    return MM_OK;
}

int mm_set_attempt_kernel(mm_ctx* C, int kind) {
    if (!C) return MM_EINVAL;
    if (kind != MM_ATTEMPT_AUTO && kind != MM_ATTEMPT_PASSES && kind != 2 && kind != 4 && kind != 8 && kind != 16)
        return fail(C, MM_EINVAL, "attempt kernel must be MM_ATTEMPT_AUTO, MM_ATTEMPT_PASSES or 2, 4, 8, 16 CTAs");
    C->attempt_kernel = kind;
    C->small_nc = -1;
    return MM_OK;
}

int mm_get_attempt_kernel(mm_ctx* C, int* single, int* cluster) {
    int rc = check_ready(C);
    if (rc) return rc;
    if (C->small_nc < 0) small_resolve(C);
    const bool one = C->small_nc > 0 && !C->neb;
    if (single) *single = one ? 1 : 0;
    if (cluster) *cluster = one ? C->small_nc : 0;
    return MM_OK;
}

int mm_set_field(mm_ctx* C, int sim, const double H[3]) {
    if (!C || !H) return MM_EINVAL;
    if (sim < 0 || sim >= (int)C->sims.size()) return fail(C, MM_EINVAL, "bad sim id");
    SimHost& s = C->sims[sim];
    for (int i = 0; i < 3; ++i) {
        s.mat.H[i] = H[i];
        s.d.H[i] = H[i];
    }
    replan(s);
    C->small_nc = -1;           // term flags may change: resolve the attempt path again
    if (C->finalized) {
        CK(cudaMemcpyAsync(&C->desc_d[sim], &s.d, sizeof(SimDesc), cudaMemcpyHostToDevice, C->stream));
        CK(cudaStreamSynchronize(C->stream));
    }
    return MM_OK;
}

int mm_set_cell_params(mm_ctx* C, int sim, const double* A_cells, const double* D_cells) {
    if (!C) return MM_EINVAL;
    if (sim < 0 || sim >= (int)C->sims.size()) return fail(C, MM_EINVAL, "bad sim id");
    if (C->finalized) return fail(C, MM_EINVAL, "mm_set_cell_params after mm_precompute_demag");
    SimHost& s = C->sims[sim];
    const size_t n = (size_t)s.d.ncells;
    if (!A_cells && !D_cells) {
        s.AD.clear();
    } else {
        std::vector<double> ad(2 * n);
        for (size_t i = 0; i < n; ++i) {
            ad[i] = A_cells ? A_cells[i] : s.mat.A;
            ad[n + i] = D_cells ? D_cells[i] : s.mat.D;
            if (!std::isfinite(ad[i]) || !std::isfinite(ad[n + i]))
                return fail(C, MM_EINVAL, "per-cell A and D must be finite");
        }
        s.AD.swap(ad);
    }
    replan(s);
    return MM_OK;
}

int mm_set_spin_torque(mm_ctx* C, int sim, const double u[3], double beta, double a_J, double b_J,
                       const double p[3]) {
    if (!C || !u || !p) return fail(C, MM_EINVAL, "NULL argument");
    if (sim < 0 || sim >= (int)C->sims.size()) return fail(C, MM_EINVAL, "bad sim id");
    bool fin = std::isfinite(beta) && std::isfinite(a_J) && std::isfinite(b_J);
    for (int i = 0; i < 3; ++i) fin = fin && std::isfinite(u[i]) && std::isfinite(p[i]);
    if (!fin) return fail(C, MM_EINVAL, "mm_set_spin_torque: non-finite argument");
    const double pn = std::sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    if ((a_J != 0.0 || b_J != 0.0) && !(pn > 0.0)) return fail(C, MM_EINVAL, "polarisation p is zero");
    SimHost& s = C->sims[sim];
    const bool before = batch_ext(C);
    for (int i = 0; i < 3; ++i) {
        s.d.u_stt[i] = u[i];
        s.d.p[i] = p[i];
    }
    s.d.beta = beta;
    s.d.aJ = a_J;
    s.d.bJ = b_J;
    replan(s);
    C->small_nc = -1;           // the torques decide whether the single-launch attempts apply
    if (C->finalized) {
        if (batch_ext(C) != before) drop_graphs(C);
        CK(cudaMemcpyAsync(&C->desc_d[sim], &s.d, sizeof(SimDesc), cudaMemcpyHostToDevice, C->stream));
        CK(cudaStreamSynchronize(C->stream));
    }
    return MM_OK;
}

int mm_precompute_demag(mm_ctx* C) {
    if (!C) return MM_EINVAL;
    if (C->finalized) return fail(C, MM_EINVAL, "already finalised");
    if (C->sims.empty()) return fail(C, MM_EINVAL, "no simulations");
    CK(cudaSetDevice(C->device));
    const bool f32 = C->precision == MM_F32;
    // geometries
    std::map<std::tuple<int, int, int, double, double, double>, int> gmap;
    for (SimHost& s : C->sims) {
        auto key = std::make_tuple(s.mesh.nx, s.mesh.ny, s.mesh.nz, s.mesh.dx, s.mesh.dy, s.mesh.dz);
        auto it = gmap.find(key);
        if (it == gmap.end()) {
            Geom g;
            g.nx = s.mesh.nx; g.ny = s.mesh.ny; g.nz = s.mesh.nz;
            g.dx = s.mesh.dx; g.dy = s.mesh.dy; g.dz = s.mesh.dz;
            gmap[key] = (int)C->geoms.size();
            C->geoms.push_back(g);
            it = gmap.find(key);
        }
        s.geom = it->second;
        if (s.d.flags & F_DEMAG) C->geoms[s.geom].demag = true;
    }
    // tensor and octant offsets
    for (size_t gi = 0; gi < C->geoms.size(); ++gi) {
        Geom& g = C->geoms[gi];
        g.oct_off = C->oct_elems;
        C->oct_elems += 6LL * g.nx * g.ny * g.nz;
        if (g.demag) {
            for (SimHost& s : C->sims)
                if (s.geom == (int)gi) {
                    g.tens_off = C->tens_elems;   // a multiple of 4 elements: 16-byte vector loads
                    C->tens_elems += (plan_tens_elems(s.d) + 3) & ~3LL;
                    break;
                }
        }
    }
    // per-simulation layout and work items (tile shapes were fixed by plan_geometry)
    PlanItems& P = C->plan;
    const size_t vsz = 2 * C->esz;
    for (size_t i = 0; i < C->sims.size(); ++i) {
        SimHost& s = C->sims[i];
        SimDesc& d = s.d;
        d.off = C->total_elems;
        C->total_elems += 3LL * d.ncells;
        d.tens_off = C->geoms[s.geom].tens_off;
        if (d.flags & F_MSARR) { d.ms_off = C->ms_elems; C->ms_elems += d.ncells; }
        if (!s.AD.empty()) { d.cell_off = C->cell_elems; C->cell_elems += 2LL * d.ncells; }
        if (d.flags & F_DEMAG) {
            // 4-element (32-byte) aligned, so every Ty-wide run of Ty >= 2 values takes 16-byte copies
            d.spec_off = (C->spec_elems + 3) & ~3LL;
            C->spec_elems = d.spec_off + plan_spec_elems(d);
        }
        else d.spec_off = 0;
        const int g = plan_uses_yzc(d) ? plan_yzc_list(d, C->precision == MM_F32) : 0;
        C->yzcl.push_back(g);
        C->xb.push_back((int)P.x.size());
        C->y13b.push_back((int)P.y13.size());
        C->zb.push_back((int)P.z.size());
        C->y2b.push_back((int)P.y2.size());
        C->yzcb.push_back((int)P.yzc[g].size());
        C->cellb.push_back((int)P.cell.size());
        plan_items(d, (int)i, vsz, P);
        C->cellc.push_back((int)P.cell.size() - C->cellb.back());
        C->xc.push_back((int)P.x.size() - C->xb.back());
        C->y13c.push_back((int)P.y13.size() - C->y13b.back());
        C->zc.push_back((int)P.z.size() - C->zb.back());
        C->y2c.push_back((int)P.y2.size() - C->y2b.back());
        C->yzcc.push_back((int)P.yzc[g].size() - C->yzcb.back());
    }
    int rc = validate_items(C);
    if (rc) return rc;
    // device memory
    const size_t sb = (size_t)C->total_elems * C->esz;
    if ((rc = dalloc(C, &C->m, sb))) return rc;
    if ((rc = dalloc(C, &C->ybuf, sb))) return rc;
    for (int j = 0; j < 7; ++j) if ((rc = dalloc(C, &C->k[j], sb))) return rc;
    if ((rc = dalloc(C, &C->errp, sb))) return rc;
    if ((rc = dalloc(C, &C->spec, (size_t)C->spec_elems * 2 * C->esz))) return rc;
    if ((rc = dalloc(C, &C->Msd, (size_t)C->ms_elems * C->esz))) return rc;
    if ((rc = dalloc(C, &C->cellp, (size_t)C->cell_elems * C->esz))) return rc;
    if ((rc = dalloc(C, &C->tens, (size_t)C->tens_elems * C->esz))) return rc;
    CK(cudaMemsetAsync(C->tens, 0, (size_t)C->tens_elems * C->esz, C->stream));   // padding of blocked tensors
    if ((rc = dalloc(C, (void**)&C->oct, (size_t)C->oct_elems * 8))) return rc;
    if ((rc = dalloc(C, &C->twd, (size_t)MM_TW_ENTRIES * 16))) return rc;
    if ((rc = dalloc(C, &C->twf, (size_t)MM_TW_ENTRIES * 8))) return rc;
    if ((rc = dalloc(C, &C->twdd, (size_t)MM_TW_ENTRIES * 16))) return rc;
    if ((rc = dalloc(C, (void**)&C->kvec_dev, 7 * sizeof(void*)))) return rc;
    if ((rc = dalloc(C, (void**)&C->desc_d, C->sims.size() * sizeof(SimDesc)))) return rc;
    if ((rc = dalloc(C, (void**)&C->state_d, C->sims.size() * sizeof(SimState)))) return rc;
    if ((rc = dalloc(C, (void**)&C->flag_d, 16))) return rc;
    if ((rc = dalloc(C, (void**)&C->status_d, 16))) return rc;
    if ((rc = dalloc(C, (void**)&C->diag_d, 16))) return rc;
    auto up_items = [&](WorkItem** dst, const std::vector<WorkItem>& v) -> int {
        int r = dalloc(C, (void**)dst, std::max<size_t>(1, v.size()) * sizeof(WorkItem));
        if (r) return r;
        if (!v.empty())
            CK(cudaMemcpyAsync(*dst, v.data(), v.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, C->stream));
        return MM_OK;
    };
    if ((rc = up_items(&C->xi, P.x))) return rc;
    if ((rc = up_items(&C->y13i, P.y13))) return rc;
    if ((rc = up_items(&C->zi, P.z))) return rc;
    if ((rc = up_items(&C->y2i, P.y2))) return rc;
    if ((rc = up_items(&C->celli, P.cell))) return rc;
    for (int li = 0; li < kYzcListCount; ++li)
        if ((rc = up_items(&C->yzci[li], P.yzc[li]))) return rc;
    CK(cudaMemcpyAsync(C->kvec_dev, C->k, 7 * sizeof(void*), cudaMemcpyHostToDevice, C->stream));
    CK(cudaMemsetAsync(C->spec, 0, (size_t)C->spec_elems * 2 * C->esz, C->stream));
    CK(cudaMemsetAsync(C->m, 0, sb, C->stream));
    CK(cudaMemsetAsync(C->ybuf, 0, sb, C->stream));
    CK(cudaMemsetAsync(C->errp, 0, sb, C->stream));
    for (int j = 0; j < 7; ++j) CK(cudaMemsetAsync(C->k[j], 0, sb, C->stream));
    // per-cell Ms
    if (C->ms_elems) {
        std::vector<double> all(C->ms_elems);
        for (const SimHost& s : C->sims)
            if (s.d.ms_off >= 0) std::copy(s.Ms.begin(), s.Ms.end(), all.begin() + s.d.ms_off);
        if (f32) {
            std::vector<float> fl(all.size());
            to_prec(all.data(), fl.data(), all.size());
            CK(cudaMemcpy(C->Msd, fl.data(), fl.size() * 4, cudaMemcpyHostToDevice));
        } else {
            CK(cudaMemcpy(C->Msd, all.data(), all.size() * 8, cudaMemcpyHostToDevice));
        }
    }
    // per-cell A and D
    if (C->cell_elems) {
        std::vector<double> all(C->cell_elems);
        for (const SimHost& s : C->sims)
            if (s.d.cell_off >= 0) std::copy(s.AD.begin(), s.AD.end(), all.begin() + s.d.cell_off);
        if (f32) {
            std::vector<float> fl(all.size());
            to_prec(all.data(), fl.data(), all.size());
            CK(cudaMemcpy(C->cellp, fl.data(), fl.size() * 4, cudaMemcpyHostToDevice));
        } else {
            CK(cudaMemcpy(C->cellp, all.data(), all.size() * 8, cudaMemcpyHostToDevice));
        }
    }
    engine_set_attributes();
    launch_twiddles(C->stream, C->twd, C->twf, C->twdd);
    upload_gauss_legendre();
    C->launches += 1;
    CK(cudaGetLastError());
    for (Geom& g : C->geoms) {
        const SimDesc* d = nullptr;
        for (const SimHost& s : C->sims) if (s.geom == (int)(&g - &C->geoms[0])) { d = &s.d; break; }
        if ((rc = precompute_geometry(C, g, *d))) return rc;
    }
    if ((rc = upload_descs(C))) return rc;
    std::vector<SimState> st(C->sims.size());
    memset(st.data(), 0, st.size() * sizeof(SimState));
    for (auto& x : st) x.rtol = 1e-6;
    if ((rc = write_states(C, st))) return rc;
    CK(cudaStreamSynchronize(C->stream));
    C->finalized = true;
    return MM_OK;
}

int mm_newell_tensor(mm_ctx* C, int sim, double* out) {
    int rc = check_ready(C);
    if (rc) return rc;
    if (sim < 0 || sim >= (int)C->sims.size() || !out) return fail(C, MM_EINVAL, "bad arguments");
    const Geom& g = C->geoms[C->sims[sim].geom];
    const long long n = (long long)g.nx * g.ny * g.nz;
    std::vector<double> oct(6 * n);
    CK(cudaMemcpyAsync(oct.data(), C->oct + g.oct_off, oct.size() * 8, cudaMemcpyDeviceToHost, C->stream));
    CK(cudaStreamSynchronize(C->stream));
    const int X = 2 * g.nx - 1, Y = 2 * g.ny - 1, Z = 2 * g.nz - 1;
    static const int odd[6] = {0, 0, 0, 3, 5, 6};
    for (int c = 0; c < 6; ++c)
        for (int k = -(g.nz - 1); k < g.nz; ++k)
            for (int j = -(g.ny - 1); j < g.ny; ++j)
                for (int i = -(g.nx - 1); i < g.nx; ++i) {
                    double sgn = 1.0;
                    if ((odd[c] & 1) && i < 0) sgn = -sgn;
                    if ((odd[c] & 2) && j < 0) sgn = -sgn;
                    if ((odd[c] & 4) && k < 0) sgn = -sgn;
                    const long long src = c * n + ((long long)std::abs(k) * g.ny + std::abs(j)) * g.nx + std::abs(i);
                    out[(((long long)c * Z + k + g.nz - 1) * Y + j + g.ny - 1) * X + i + g.nx - 1] = sgn * oct[src];
                }
    return MM_OK;
}

int mm_set_m(mm_ctx* C, int sim, const void* m, int where) {
    int rc = check_ready(C);
    if (rc) return rc;
    if (!m || sim < -1 || sim >= (int)C->sims.size()) return fail(C, MM_EINVAL, "bad arguments");
    const long long off = sim < 0 ? 0 : C->sims[sim].d.off;
    const long long n = sim < 0 ? C->total_elems : 3LL * C->sims[sim].d.ncells;
    char* dst = (char*)C->m + off * C->esz;
    if (where == MM_DEVICE) {
        CK(cudaMemcpyAsync(dst, m, n * C->esz, cudaMemcpyDeviceToDevice, C->stream));
    } else if (C->precision == MM_F32 && host_pinned(m)) {
        if ((rc = ensure_dev_stage(C, (size_t)n * 8))) return rc;
        CK(cudaMemcpyAsync(C->dev_stage, m, n * 8, cudaMemcpyHostToDevice, C->stream));
        k_convert<double, float><<<convert_blocks(n), 256, 0, C->stream>>>((const double*)C->dev_stage, (float*)dst, n);
        C->launches += 1;
        CK(cudaGetLastError());
    } else if (C->precision == MM_F32) {
        if ((rc = ensure_host_stage(C, (size_t)n * 4))) return rc;
        float* f = (float*)C->host_stage;
        convert_host((const double*)m, f, n);
        CK(cudaMemcpyAsync(dst, f, n * 4, cudaMemcpyHostToDevice, C->stream));
    } else {
        CK(cudaMemcpyAsync(dst, m, n * 8, cudaMemcpyHostToDevice, C->stream));
    }
    CK(cudaStreamSynchronize(C->stream));
    return MM_OK;
}

int mm_get_m(mm_ctx* C, int sim, void* m, int where) {
    int rc = check_ready(C);
    if (rc) return rc;
    if (!m || sim < -1 || sim >= (int)C->sims.size()) return fail(C, MM_EINVAL, "bad arguments");
    const long long off = sim < 0 ? 0 : C->sims[sim].d.off;
    const long long n = sim < 0 ? C->total_elems : 3LL * C->sims[sim].d.ncells;
    const char* src = (const char*)C->m + off * C->esz;
    if (where == MM_DEVICE) {
        CK(cudaMemcpyAsync(m, src, n * C->esz, cudaMemcpyDeviceToDevice, C->stream));
    } else if (C->precision == MM_F32 && host_pinned(m)) {
        if ((rc = ensure_dev_stage(C, (size_t)n * 8))) return rc;
        k_convert<float, double><<<convert_blocks(n), 256, 0, C->stream>>>((const float*)src, (double*)C->dev_stage, n);
        C->launches += 1;
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(m, C->dev_stage, n * 8, cudaMemcpyDeviceToHost, C->stream));
    } else if (C->precision == MM_F32) {
        if ((rc = ensure_host_stage(C, (size_t)n * 4))) return rc;
        float* f = (float*)C->host_stage;
        CK(cudaMemcpyAsync(f, src, n * 4, cudaMemcpyDeviceToHost, C->stream));
        CK(cudaStreamSynchronize(C->stream));
        convert_host(f, (double*)m, n);
    } else {
        CK(cudaMemcpyAsync(m, src, n * 8, cudaMemcpyDeviceToHost, C->stream));
    }
    CK(cudaStreamSynchronize(C->stream));
    return MM_OK;
}

int mm_rhs_eval(mm_ctx* C, int sim, const void* m_dev, void* dmdt_dev, void* heff_dev) {
    int rc = check_ready(C);
    if (rc) return rc;
    if (!m_dev || !dmdt_dev || sim < -1 || sim >= (int)C->sims.size()) return fail(C, MM_EINVAL, "bad arguments");
    Launch L = make_launch(C, sim);
    const long long adj = sim < 0 ? 0 : C->sims[sim].d.off;
    if (C->precision == MM_F32)
        engine_rhs<float>(L, 0, (const float*)m_dev, (float*)dmdt_dev, (float*)heff_dev, adj);
    else
        engine_rhs<double>(L, 0, (const double*)m_dev, (double*)dmdt_dev, (double*)heff_dev, adj);
    CK(cudaGetLastError());
    return MM_OK;
}

int mm_demag_potential(mm_ctx* C, int sim, const void* m_dev, void* hd_dev) {
    int rc = check_ready(C);
    if (rc) return rc;
    if (!m_dev || !hd_dev || sim < 0 || sim >= (int)C->sims.size()) return fail(C, MM_EINVAL, "bad arguments");
    const SimHost& S = C->sims[sim];
    const PotGeom g = pot_geometry(S.mesh.nx, S.mesh.ny, S.mesh.nz, S.mesh.dx, S.mesh.dy, S.mesh.dz);
    if (g.Px > kPotMaxP || g.Py > kPotMaxP || g.Pz > kPotMaxP)
        return fail(C, MM_EINVAL, "scalar-potential demag: padded length %d x %d x %d above %d (mesh axes <= %d cells)",
                    g.Px, g.Py, g.Pz, kPotMaxP, kPotMaxP / 2 - 1);
    const bool f32 = C->precision == MM_F32;
    const size_t cz = 2 * C->esz;             // complex value in the context precision
    mm_ctx::PotPlan* P = nullptr;
    for (auto& pp : C->pot)
        if (pp.g.nx == g.nx && pp.g.ny == g.ny && pp.g.nz == g.nz && pp.g.dx == g.dx && pp.g.dy == g.dy &&
            pp.g.dz == g.dz)
            P = &pp;
    if (!P) {
        mm_ctx::PotPlan np;
        np.g = g;
        const long long nb = pot_bins(g);
        if ((rc = dalloc(C, &np.b.Shat, 3 * nb * cz))) return rc;
        if ((rc = dalloc(C, &np.b.Mhat, 3 * nb * cz)) || (rc = dalloc(C, &np.b.U, nb * cz)) ||
            (rc = dalloc(C, &np.b.u, pot_ext_cells(g) * C->esz))) {
            void* pb[] = {np.b.Shat, np.b.Mhat, np.b.U, np.b.u};
            for (void* p : pb) if (p) cudaFree(p);
            return rc;
        }
        void* s64 = nullptr;
        if ((rc = dalloc(C, &s64, 3 * nb * 16))) {
            void* pb[] = {np.b.Shat, np.b.Mhat, np.b.U, np.b.u};
            for (void* p : pb) if (p) cudaFree(p);
            return rc;
        }
        cudaError_t e = pot_precompute(C->stream, g, np.b.Shat, f32, s64, C->twd, &C->launches);
        cudaStreamSynchronize(C->stream);
        cudaFree(s64);
        if (e != cudaSuccess) {
            void* pb[] = {np.b.Shat, np.b.Mhat, np.b.U, np.b.u};
            for (void* p : pb) if (p) cudaFree(p);
            return fail(C, MM_ECUDA, "scalar-potential kernel spectrum: %s", cudaGetErrorString(e));
        }
        C->pot.push_back(np);
        P = &C->pot.back();
    }
    const SimDesc& d = S.d;
    const void* Ms = (d.flags & F_MSARR) ? (const char*)C->Msd + d.ms_off * C->esz : nullptr;
    const void* tw = f32 ? C->twf : C->twd;
    cudaError_t e = pot_field(C->stream, P->g, P->b, f32, m_dev, Ms, d.Ms, hd_dev, tw, &C->launches);
    if (e != cudaSuccess) return fail(C, MM_ECUDA, "scalar-potential demag: %s", cudaGetErrorString(e));
    return MM_OK;
}

int mm_rhs_eval_host(mm_ctx* C, int sim, const double* m, double* dmdt, double* heff) {
    int rc = check_ready(C);
    if (rc) return rc;
    if (!m || !dmdt || sim < -1 || sim >= (int)C->sims.size()) return fail(C, MM_EINVAL, "bad arguments");
    if ((rc = ensure_scratch(C))) return rc;
    const long long n = sim < 0 ? C->total_elems : 3LL * C->sims[sim].d.ncells;
    if (C->precision == MM_F32) {
        std::vector<float> f(n);
        to_prec(m, f.data(), n);
        CK(cudaMemcpyAsync(C->sc_in, f.data(), n * 4, cudaMemcpyHostToDevice, C->stream));
        if ((rc = mm_rhs_eval(C, sim, C->sc_in, C->sc_out, heff ? C->sc_h : nullptr))) return rc;
        CK(cudaMemcpyAsync(f.data(), C->sc_out, n * 4, cudaMemcpyDeviceToHost, C->stream));
        CK(cudaStreamSynchronize(C->stream));
        for (long long i = 0; i < n; ++i) dmdt[i] = f[i];
        if (heff) {
            CK(cudaMemcpyAsync(f.data(), C->sc_h, n * 4, cudaMemcpyDeviceToHost, C->stream));
            CK(cudaStreamSynchronize(C->stream));
            for (long long i = 0; i < n; ++i) heff[i] = f[i];
        }
    } else {
        CK(cudaMemcpyAsync(C->sc_in, m, n * 8, cudaMemcpyHostToDevice, C->stream));
        if ((rc = mm_rhs_eval(C, sim, C->sc_in, C->sc_out, heff ? C->sc_h : nullptr))) return rc;
        CK(cudaMemcpyAsync(dmdt, C->sc_out, n * 8, cudaMemcpyDeviceToHost, C->stream));
        if (heff) CK(cudaMemcpyAsync(heff, C->sc_h, n * 8, cudaMemcpyDeviceToHost, C->stream));
        CK(cudaStreamSynchronize(C->stream));
    }
    return MM_OK;
}

int mm_rk45_setup(mm_ctx* C, double rtol, double t_end, double max_dmdt) {
    int rc = check_ready(C);
    if (rc) return rc;
    if (!(rtol > 0)) return fail(C, MM_EINVAL, "rtol must be > 0");
    std::vector<SimState> st;
    if ((rc = read_states(C, st))) return rc;
    for (auto& s : st) {
        s.rtol = rtol;
        s.t_end = t_end;
        s.max_dmdt = max_dmdt;
        if (s.status >= 0) s.status = 0;
    }
    return write_states(C, st);
}

int mm_reset_time(mm_ctx* C) {
    int rc = check_ready(C);
    if (rc) return rc;
    std::vector<SimState> st;
    if ((rc = read_states(C, st))) return rc;
    for (auto& s : st) {
        s.t = 0.0; s.h = 0.0; s.n_acc = 0; s.n_rej = 0; s.status = 0; s.accepted = 0;
        s.err_bits = 0; s.maxk_bits = 0;
    }
    return write_states(C, st);
}

int mm_rk45_attempts(mm_ctx* C, int n) {
    int rc = check_ready(C);
    if (rc) return rc;
    if (n < 0) return fail(C, MM_EINVAL, "n < 0");
    return launch_attempts(C, n);
}

int mm_rk45_step(mm_ctx* C, int* n_acc, int* n_rej) {
    int rc = check_ready(C);
    if (rc) return rc;
    std::vector<SimState> st;
    if ((rc = read_states(C, st))) return rc;
    std::vector<long long> acc0(st.size()), rej0(st.size());
    for (size_t i = 0; i < st.size(); ++i) { acc0[i] = st[i].n_acc; rej0[i] = st[i].n_rej; }
    for (int it = 0; it < 1000; ++it) {
        bool any = false;
        for (auto& s : st) any |= s.status == 0;
        if (!any) break;
        if ((rc = launch_attempts(C, 1))) return rc;
        if ((rc = read_states(C, st))) return rc;
        if ((rc = first_error(C, st))) return rc;
        bool changed = false;
        for (auto& s : st)
            if (s.status == 0 && s.accepted) { s.status = 3; changed = true; }   // pause until all accepted
        if (changed && (rc = write_states(C, st))) return rc;
    }
    long long a = 0, r = 0;
    for (size_t i = 0; i < st.size(); ++i) {
        if (st[i].status == 3) st[i].status = 0;
        a += st[i].n_acc - acc0[i];
        r += st[i].n_rej - rej0[i];
    }
    if ((rc = write_states(C, st))) return rc;
    if (n_acc) *n_acc = (int)a;
    if (n_rej) *n_rej = (int)r;
    return MM_OK;
}

int mm_relax(mm_ctx* C, double rtol, double t_end, double max_dmdt, long long max_steps, int sync_every,
             long long* done) {
    int rc = check_ready(C);
    if (rc) return rc;
    if ((rc = mm_rk45_setup(C, rtol, t_end, max_dmdt))) return rc;
    if (sync_every < 1) sync_every = 1;
    long long att = 0;
    std::vector<SimState> st;
    while (att < max_steps) {
        const long long n = std::min<long long>(sync_every, max_steps - att);
        if ((rc = launch_attempts(C, n))) return rc;
        att += n;
        if ((rc = read_states(C, st))) return rc;
        if ((rc = first_error(C, st))) return rc;
        bool live = false;
        for (auto& s : st) live |= s.status == 0;
        if (!live) break;
    }
    if (done) *done = att;
    return MM_OK;
}

int mm_minimize(mm_ctx* C, double max_dmdt, long long max_steps, int sync_every, long long* steps_done,
                int* converged) {
    int rc = check_ready(C);
    if (rc) return rc;
    if (C->neb) return fail(C, MM_EINVAL, "mm_minimize: not in a context with NEB chains");
    if (!(max_dmdt >= 0.0) || max_steps < 0) return fail(C, MM_EINVAL, "mm_minimize: bad arguments");
    if (sync_every < 1) sync_every = 1;
    if ((rc = sd_prepare(C))) return rc;
    // fresh state: tau_0 at the first step, zero history
    std::vector<SdState> h(C->sims.size());
    for (size_t i = 0; i < C->sims.size(); ++i) {
        const mm_material& mt = C->sims[i].mat;
        SdState z;
        memset(&z, 0, sizeof(z));
        const double gt = mt.gamma / (1.0 + mt.alpha * mt.alpha);
        z.dmdt_scale = gt * (mt.precession ? std::sqrt(1.0 + mt.alpha * mt.alpha) : mt.alpha);
        z.stop_dmdt = max_dmdt;
        z.max_dmdt = HUGE_VAL;
        h[i] = z;
    }
    const size_t sb = (size_t)C->total_elems * C->esz;
    CK(cudaMemcpyAsync(C->sd_d, h.data(), h.size() * sizeof(SdState), cudaMemcpyHostToDevice, C->stream));
    CK(cudaMemsetAsync(C->sd_mprev, 0, sb, C->stream));
    CK(cudaMemsetAsync(C->sd_g, 0, sb, C->stream));
    long long done = 0;
    while (done < max_steps) {
        const long long n = std::min<long long>(sync_every, max_steps - done);
        for (long long i = 0; i < n; ++i) CK(cudaGraphLaunch(C->sd_exec, C->stream));
        C->launches += n * C->sd_graph_kernels;
        done += n;
        CK(cudaMemcpyAsync(h.data(), C->sd_d, h.size() * sizeof(SdState), cudaMemcpyDeviceToHost, C->stream));
        CK(cudaStreamSynchronize(C->stream));
        bool live = false;
        for (size_t i = 0; i < h.size(); ++i) {
            if (h[i].status < 0) return fail(C, MM_ENAN, "mm_minimize: simulation %zu: non-finite field", i);
            live |= h[i].status == 0;
        }
        if (!live) break;
    }
    long long kmax = 0;
    bool all = true;
    for (const SdState& s : h) {
        kmax = std::max(kmax, s.k);
        all &= s.status == 2;
    }
    if (steps_done) *steps_done = kmax;
    if (converged) *converged = all ? 1 : 0;
    return MM_OK;
}

int mm_rk4(mm_ctx* C, double h, long long n_steps, int cayley) {
    int rc = check_ready(C);
    if (rc) return rc;
    if (C->neb) return fail(C, MM_EINVAL, "mm_rk4: not in a context with NEB chains");
    if (!(h > 0.0) || std::isinf(h) || n_steps < 0 || (cayley != 0 && cayley != 1))
        return fail(C, MM_EINVAL, "mm_rk4: bad arguments");
    if (cayley)
        for (const SimHost& s : C->sims)
            if (s.d.eflags & (E_STT | E_SOT))
                return fail(C, MM_EINVAL, "mm_rk4: the Cayley scheme takes f from H_eff; spin torques need cayley = 0");
    if ((rc = c4_prepare(C, h, cayley))) return rc;
    for (long long i = 0; i < n_steps; ++i) CK(cudaGraphLaunch(C->c4_exec, C->stream));
    C->launches += n_steps * C->c4_graph_kernels;
    CK(cudaStreamSynchronize(C->stream));
    return MM_OK;
}

int mm_minimize_info(mm_ctx* C, int sim, long long* steps, double* tau, double* max_dmdt, int* status) {
    if (!C) return MM_EINVAL;
    if (sim < 0 || sim >= (int)C->sims.size()) return fail(C, MM_EINVAL, "bad sim id");
    if (!C->sd_d) return fail(C, MM_EINVAL, "mm_minimize_info: mm_minimize has not run");
    SdState s;
    CK(cudaMemcpyAsync(&s, C->sd_d + sim, sizeof(s), cudaMemcpyDeviceToHost, C->stream));
    CK(cudaStreamSynchronize(C->stream));
    if (steps) *steps = s.k;
    if (tau) *tau = s.tau;
    if (max_dmdt) *max_dmdt = s.max_dmdt;
    if (status) *status = s.status;
    return MM_OK;
}

int mm_get_status(mm_ctx* C, int sim, mm_status* out) {
    int rc = check_ready(C);
    if (rc) return rc;
    if (!out || sim < 0 || sim >= (int)C->sims.size()) return fail(C, MM_EINVAL, "bad arguments");
    SimState s;
    CK(cudaMemcpyAsync(&s, C->state_d + sim, sizeof(s), cudaMemcpyDeviceToHost, C->stream));
    CK(cudaStreamSynchronize(C->stream));
    out->t = s.t; out->h = s.h; out->err = s.err; out->max_dmdt = s.maxk;
    out->n_accepted = s.n_acc; out->n_rejected = s.n_rej;
    out->status = s.status; out->pad = 0;
    return MM_OK;
}

int mm_get_checkpoint(mm_ctx* C, int sim, mm_checkpoint* out) {
    int rc = check_ready(C);
    if (rc) return rc;
    if (!out || sim < 0 || sim >= (int)C->sims.size()) return fail(C, MM_EINVAL, "bad arguments");
    SimState s;
    CK(cudaMemcpyAsync(&s, C->state_d + sim, sizeof(s), cudaMemcpyDeviceToHost, C->stream));
    CK(cudaStreamSynchronize(C->stream));
    out->t = s.t; out->h = s.h; out->t_end = s.t_end; out->rtol = s.rtol; out->max_dmdt = s.max_dmdt;
    out->n_accepted = s.n_acc; out->n_rejected = s.n_rej;
    out->status = s.status; out->pad = 0;
    return MM_OK;
}

int mm_set_checkpoint(mm_ctx* C, int sim, const mm_checkpoint* in) {
    int rc = check_ready(C);
    if (rc) return rc;
    if (!in || sim < 0 || sim >= (int)C->sims.size()) return fail(C, MM_EINVAL, "bad arguments");
    const bool st_ok = in->status == 0 || in->status == 1 || in->status == 2 || in->status == MM_ENAN ||
                       in->status == MM_ESTEP;
    if (!(in->rtol > 0.0) || !(in->h >= 0.0) || std::isinf(in->h) || !std::isfinite(in->t) ||
        !(in->t_end >= 0.0) || std::isinf(in->t_end) || !(in->max_dmdt >= 0.0) || in->n_accepted < 0 ||
        in->n_rejected < 0 || !st_ok)
        return fail(C, MM_EINVAL, "mm_set_checkpoint: invalid checkpoint");
    SimState s;
    memset(&s, 0, sizeof(s));   // reductions start from zero, as after the controller of an attempt
    s.t = in->t; s.h = in->h; s.t_end = in->t_end; s.rtol = in->rtol; s.max_dmdt = in->max_dmdt;
    s.n_acc = in->n_accepted; s.n_rej = in->n_rejected;
    s.status = in->status;
    CK(cudaMemcpyAsync(C->state_d + sim, &s, sizeof(s), cudaMemcpyHostToDevice, C->stream));
    CK(cudaStreamSynchronize(C->stream));
    return MM_OK;
}

int mm_energy(mm_ctx* C, int sim, double E[7]) {
    int rc = check_ready(C);
    if (rc) return rc;
    if (!E || sim < -1 || sim >= (int)C->sims.size()) return fail(C, MM_EINVAL, "bad arguments");
    CK(cudaMemset2DAsync(&C->state_d[0].E[0], sizeof(SimState), 0, 8 * sizeof(double), C->sims.size(), C->stream));
    Launch L = make_launch(C, sim);
    if (C->precision == MM_F32)
        engine_rhs<float>(L, MODE_ENERGY, (const float*)C->m, nullptr, nullptr, 0);
    else
        engine_rhs<double>(L, MODE_ENERGY, (const double*)C->m, nullptr, nullptr, 0);
    CK(cudaGetLastError());
    std::vector<SimState> st;
    if ((rc = read_states(C, st))) return rc;
    const int s = sim < 0 ? 0 : sim;
    double tot = 0;
    for (int i = 0; i < 6; ++i) { E[i] = st[s].E[i]; tot += E[i]; }
    E[6] = tot;
    return MM_OK;
}

int mm_neb_setup(mm_ctx* C, int first, int n, double k_spring) {
    int rc = check_ready(C);
    if (rc) return rc;
    if (n < 3 || first < 0 || first + n > (int)C->sims.size()) return fail(C, MM_EINVAL, "bad chain range");
    const SimDesc& d0 = C->sims[first].d;
    for (int i = first; i < first + n; ++i) {
        const SimDesc& d = C->sims[i].d;
        if (d.nx != d0.nx || d.ny != d0.ny || d.nz != d0.nz || d.group_begin >= 0)
            return fail(C, MM_EINVAL, "chain images must share one mesh and belong to no other chain");
    }
    for (int i = first; i < first + n; ++i) {
        SimDesc& d = C->sims[i].d;
        d.group_begin = first;
        d.group_end = first + n;
        d.neb_index = i - first;
        d.k_spring = k_spring;
    }
    for (const SimHost& s : C->sims)
        if (s.d.group_begin < 0) return fail(C, MM_EINVAL, "every simulation of a NEB context must be in a chain");
    if (!C->heff) {
        const size_t sb = (size_t)C->total_elems * C->esz;
        if ((rc = dalloc(C, &C->heff, sb))) return rc;
        if ((rc = dalloc(C, &C->tau, sb))) return rc;
        CK(cudaMemset(C->heff, 0, sb));
        CK(cudaMemset(C->tau, 0, sb));
    }
    C->neb = true;
    return upload_descs(C);
}

int mm_neb_relax(mm_ctx* C, double rtol, long long n_steps, double* energies) {
    int rc = check_ready(C);
    if (rc) return rc;
    if (!C->neb) return fail(C, MM_EINVAL, "call mm_neb_setup first");
    if ((rc = mm_rk45_setup(C, rtol, 0.0, 0.0))) return rc;
    if ((rc = launch_attempts(C, n_steps))) return rc;
    std::vector<SimState> st;
    if ((rc = read_states(C, st))) return rc;
    if ((rc = first_error(C, st))) return rc;
    if (energies) {
        CK(cudaMemset2DAsync(&C->state_d[0].E[0], sizeof(SimState), 0, 8 * sizeof(double), C->sims.size(),
                             C->stream));
        Launch L = make_launch(C, -1);
        if (C->precision == MM_F32)
            engine_rhs<float>(L, MODE_ENERGY, (const float*)C->m, nullptr, nullptr, 0);
        else
            engine_rhs<double>(L, MODE_ENERGY, (const double*)C->m, nullptr, nullptr, 0);
        CK(cudaGetLastError());
        if ((rc = read_states(C, st))) return rc;
        for (size_t i = 0; i < st.size(); ++i) {
            double t = 0;
            for (int j = 0; j < 6; ++j) t += st[i].E[j];
            energies[i] = t;
        }
    }
    return MM_OK;
}

int mm_profile_attempts(mm_ctx* C, int reps, double* ms, long long* counts) {
    int rc = check_ready(C);
    if (rc) return rc;
    if (reps < 1 || !ms || !counts) return fail(C, MM_EINVAL, "bad arguments");
    ProfileHook H;
    H.stream = C->stream;
    H.cap = 64 * reps + 2;
    std::vector<cudaEvent_t> ev(H.cap);
    std::vector<int> kinds(H.cap, -1);
    for (auto& e : ev) CK(cudaEventCreate(&e));
    H.ev = ev.data();
    H.kinds = kinds.data();
    Launch L = make_launch(C, -1);
    L.hook = &H;
    RkBuffers B;
    B.m = C->m; B.ybuf = C->ybuf; B.kvec_dev = C->kvec_dev; B.errp = C->errp;
    for (int j = 0; j < 7; ++j) B.kvec[j] = C->k[j];
    B.heff = C->heff;
    B.tau = C->tau;
    H.mark(-1);
    for (int r = 0; r < reps; ++r) {
        if (C->neb) {
            if (C->precision == MM_F32) engine_neb_attempt<float>(L, B); else engine_neb_attempt<double>(L, B);
        } else {
            if (C->precision == MM_F32) engine_attempt<float>(L, B); else engine_attempt<double>(L, B);
        }
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(C->stream));
    for (int k = 0; k < KIND_COUNT; ++k) { ms[k] = 0.0; counts[k] = 0; }
    for (int i = 1; i < H.used; ++i) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, ev[i - 1], ev[i]));
        if (kinds[i] >= 0 && kinds[i] < KIND_COUNT) { ms[kinds[i]] += t; counts[kinds[i]] += 1; }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    return MM_OK;
}

int mm_debug_bounded_wait(mm_ctx* C, long long spins) {
    if (spins < 0 || spins > MM_MAX_WAIT_SPINS)
        return fail(C, MM_EINVAL, "mm_debug_bounded_wait: spins must be in [0, %lld]", (long long)MM_MAX_WAIT_SPINS);
    int rc = check_ready(C);
    if (rc) return rc;
    CK(cudaMemsetAsync(C->flag_d, 0, 16, C->stream));
    CK(cudaMemsetAsync(C->status_d, 0, 16, C->stream));
    engine_bounded_wait(C->stream, C->flag_d, spins, C->status_d);
    C->launches += 1;
    CK(cudaGetLastError());
    int st = 0;
    CK(cudaMemcpyAsync(&st, C->status_d, sizeof(int), cudaMemcpyDeviceToHost, C->stream));
    CK(cudaStreamSynchronize(C->stream));
    if (st == MM_ETIMEOUT) return fail(C, MM_ETIMEOUT, "bounded device wait ran out after %lld polls", spins);
    return MM_OK;
}

long long mm_kernel_launches(const mm_ctx* C) { return C ? C->launches : 0; }

}  // extern "C"

// Error message of calls that have no context (mm_last_error(NULL)).
void mm_internal_set_error(const char* msg) { snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }
