// Host-side planning of one simulation: padded FFT lengths, tile shapes and
// the work items of every pass.  Shared by the context API and the
// allocation-free entry point so both lay out a simulation the same way.
#pragma once
#include <algorithm>
#include <cmath>
#include <vector>

#include "mm_kernels.cuh"

namespace mm {

inline int plan_ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

inline int plan_pow2floor(int v) {
    int p = 1;
    while (p * 2 <= v) p *= 2;
    return p;
}

// padded FFT length: the smallest power of two >= 2n - 1 (1 for n == 1 unless min2)
inline int plan_pad_len(int n, bool min2) {
    if (n <= 1) return min2 ? 2 : 1;
    int p = 1;
    while (p < 2 * n - 1) p <<= 1;
    return p;
}


// Tile shapes and schedules an autotuner may set per simulation; 0 keeps the
// fixed rule of plan_geometry / plan_yzc_list / plan_wide_threads.
//   Ty          kx block width (power of two, 1..32)
//   Rx          rows per x-pass CTA (1..ny)
//   x_threads   threads of an x-pass CTA (multiple of 32; launch-wide)
//   col_threads threads of a column-pass CTA outside the cluster pass (launch-wide)
//   col_group   cluster-pass column register groups: 1 16-point, 2 32-point
//   col_occ     cluster-pass CTAs per SM its kernel is built for: 3 or 4 (FP32, up
//               to kYzcOcc3MaxPlanes planes; fewer registers a thread, 8-point
//               column groups at 4), else the rule (2)
//   x_stage     1: the x-inverse pass stages its tile's state rows (and their +-y,
//               +-z neighbours) in shared memory by bulk copies; else the rule (loads)
struct Tuning {
    int Ty = 0, Rx = 0, x_threads = 0, col_threads = 0, col_group = 0, col_occ = 0, x_stage = 0;
};

// Fill the padded sizes, tensor bins and tile shapes of d from d.nx, d.ny, d.nz
// (the rule, unless the tuning t sets a value).
//   Rx : rows per x-pass CTA, 3 * Rx * padded_len(Kx) <= 4096 complex values per
//        buffer (two buffers), Rx <= ny; tiles never cross a plane
//   Ty : kx block width (power of two, <= 32): Py * Ty <= 4096 (FP32) / 2048 (FP64)
inline void plan_geometry(SimDesc& d, bool f32, const Tuning& t = Tuning()) {
    d.Px = plan_pad_len(d.nx, true);
    d.Py = plan_pad_len(d.ny, false);
    d.Pz = plan_pad_len(d.nz, false);
    d.lPx = plan_ilog2(d.Px);
    d.lPy = plan_ilog2(d.Py);
    d.lPz = plan_ilog2(d.Pz);
    d.Kx = d.Px / 2 + 1;
    d.Pyh = d.Py / 2 + 1;
    d.Pzh = d.Pz / 2 + 1;
    d.ncomp = d.Pz > 1 ? 6 : 4;
    const int rows = d.ny * d.nz;
    // small meshes: keep at least ~rows/64 CTAs (one row each for <= 64 rows) so a
    // lone small simulation still spreads over many SMs
    const int rcap = std::max(1, (rows + 63) / 64);
    d.Rx = std::max(1, std::min(std::min(std::min(rows, d.ny), rcap), 4096 / (3 * padded_len(d.Kx))));
    const int EB = f32 ? 4096 : 2048;
    const int kcap = std::min(32, std::max(1, plan_pow2floor(std::max(1, d.Kx / 8))));
    d.Ty = std::min(kcap, plan_pow2floor(std::max(1, EB / d.Py)));
    if (t.Rx > 0) d.Rx = std::min(t.Rx, d.ny);
    if (t.Ty > 0) d.Ty = plan_pow2floor(std::min(t.Ty, 32));
    d.lTy = plan_ilog2(d.Ty);
    d.NBx = (d.Kx + d.Ty - 1) >> d.lTy;
    d.colgroup = (t.col_group == 1 || t.col_group == 2) ? t.col_group : 0;
    d.yzcocc = (t.col_occ == 3 || t.col_occ == 4) ? t.col_occ : 0;
    d.flags = (d.flags & ~F_XSTAGE) | (t.x_stage == 1 ? F_XSTAGE : 0);
}

template <typename T>
inline void plan_fill_coef(Coef<T>& c, const SimDesc& d) {
    const double mu0 = 4e-7 * 3.14159265358979323846;
    c.Ms = (T)d.Ms;
    c.mu0 = (T)mu0;
    c.inv_u = d.Ms > 0.0 ? (T)(1.0 / (mu0 * d.Ms)) : (T)0;
    c.ex[0] = (T)(1.0 / (d.dx * d.dx));
    c.ex[1] = (T)(1.0 / (d.dy * d.dy));
    c.ex[2] = (T)(1.0 / (d.dz * d.dz));
    c.dm[0] = (T)(1.0 / d.dx);
    c.dm[1] = (T)(1.0 / d.dy);
    c.cA = (T)(2.0 * d.A);
    c.cD = (T)d.D;
    c.cK = (T)(2.0 * d.Ku);
    c.cC = (T)(4.0 * d.Kc);
    for (int i = 0; i < 3; ++i) { c.u[i] = (T)d.u[i]; c.H[i] = (T)d.H[i]; }
    c.gt = (T)(d.gamma / (1.0 + d.alpha * d.alpha));
    c.agt = (T)(d.alpha * d.gamma / (1.0 + d.alpha * d.alpha));
    c.pad = (T)0;
}

// Derive the term flags and both coefficient sets of d from its FP64 material
// parameters; call again after any parameter (the applied field) changes.
// dmi_interfacial: the material's DMI kind is interfacial.
inline void plan_coefficients(SimDesc& d, bool dmi_interfacial) {
    d.flags &= ~(F_DMI | F_EX | F_UNI | F_CUB);
    if (dmi_interfacial && d.D != 0.0) d.flags |= F_DMI;
    if (d.A != 0.0) d.flags |= F_EX;
    if (d.Ku != 0.0) d.flags |= F_UNI;
    if (d.Kc != 0.0) d.flags |= F_CUB;
    plan_fill_coef(d.cd, d);
    plan_fill_coef(d.cf, d);
}

template <typename T>
inline void plan_fill_ext(ExtCoef<T>& c, const SimDesc& d) {
    c.A = (T)d.A;
    c.D = (T)d.D;
    c.dinv_z = (T)(1.0 / d.dz);
    c.gu[0] = (T)(d.u_stt[0] / (2.0 * d.dx));
    c.gu[1] = (T)(d.u_stt[1] / (2.0 * d.dy));
    c.gu[2] = (T)(d.u_stt[2] / (2.0 * d.dz));
    c.beta = (T)d.beta;
    c.aJ = (T)d.aJ;
    c.bJ = (T)d.bJ;
    c.alpha = (T)d.alpha;
    c.inv_q = (T)(1.0 / (1.0 + d.alpha * d.alpha));
    const double pn = std::sqrt(d.p[0] * d.p[0] + d.p[1] * d.p[1] + d.p[2] * d.p[2]);
    for (int i = 0; i < 3; ++i) c.p[i] = pn > 0.0 ? (T)(d.p[i] / pn) : (T)0;
}

// The extended terms of d (after plan_coefficients): eflags, F_EXT and, for an
// extended simulation, F_EX / F_DMI with the per-cell constants taken into
// account, and both extended coefficient sets.  has_cells: per-cell A and D
// are given; a_any / d_any: some per-cell A / D is non-zero.
inline void plan_extended(SimDesc& d, bool has_cells, bool a_any, bool d_any) {
    d.flags &= ~F_EXT;
    d.eflags = 0;
    if (has_cells) d.eflags |= E_CELL;
    if (d.u_stt[0] != 0.0 || d.u_stt[1] != 0.0 || d.u_stt[2] != 0.0) d.eflags |= E_STT;
    if (d.aJ != 0.0 || d.bJ != 0.0) d.eflags |= E_SOT;
    if (d.eflags != 0 || d.dmi_kind >= 2) d.flags |= F_EXT;
    if (d.flags & F_EXT) {
        const bool ex = d.A != 0.0 || (has_cells && a_any);
        const bool dmi = d.dmi_kind != 0 && (d.D != 0.0 || (has_cells && d_any));
        d.flags = (d.flags & ~(F_EX | F_DMI)) | (ex ? F_EX : 0) | (dmi ? F_DMI : 0);
    }
    plan_fill_ext(d.xd, d);
    plan_fill_ext(d.xf, d);
}

// Films with 2..kMaxClusterPlanes planes run the cluster-fused y/z pass, which
// reads its tensor in a blocked layout (plan_tens_elems).
inline bool plan_uses_yzc(const SimDesc& d) { return d.Pz > 1 && d.Py > 1 && d.nz <= kMaxClusterPlanes; }

// Cluster-pass work lists, one per (plane count nz, register-group width, CTAs
// per SM): list nz + kYzcLists * wide + 2 kYzcLists * occ3.  FP32 columns of
// 2^5, 2^9 or 2^13 points run
// with 32-point register groups (their schedule then holds exactly one
// 32-point group: (5), (5,4), (5,4,4)); every other length with 16-point
// groups, whose schedule is the same or better (two unrolled 32-point groups
// per direction no longer fit the instruction cache: 1024-point columns
// measured faster as (4,3,3) than as (5,5)).
inline int plan_yzc_list(const SimDesc& d, bool f32) {
    const bool wide = d.colgroup ? d.colgroup == 2 : f32 && (d.lPy == 5 || d.lPy == 9 || d.lPy == 13);
    const int occ = d.yzcocc == 3 ? 1 : d.yzcocc == 4 ? 2 : 0;
    return d.nz + kYzcLists * ((wide ? 1 : 0) + 2 * occ);
}
inline int plan_yzc_nz(int li) { return li % kYzcLists; }
inline bool plan_yzc_wide(int li) { return ((li / kYzcLists) & 1) != 0; }
// CTAs per SM of list li's kernel build (2: the rule's)
inline int plan_yzc_occ(int li) { return 2 + li / (2 * kYzcLists); }

// Elements of a geometry's stored tensor:
//   standard [ncomp][Pz/2+1][Py/2+1][Kx];
//   blocked (cluster pass) [NBx][Py/2+1][Ty][qp], entry q = 6 dz + c for the
//   plane offsets dz = 0..nz-1, so the values one column of one ky row needs
//   are contiguous.
inline long long plan_tens_elems(const SimDesc& d) {
    if (plan_uses_yzc(d)) return (long long)d.NBx * d.Pyh * d.Ty * yzc_qp(d.nz);
    return (long long)d.ncomp * d.Pzh * d.Pyh * d.Kx;
}

inline long long plan_spec_elems(const SimDesc& d) { return 3LL * d.nz * d.NBx * d.Py * d.Ty; }

// x-inverse shared memory: two FFT buffers of 3*Rx padded rows, then (F_XSTAGE)
// the staged state rows.
inline size_t plan_xinv_smem(const SimDesc& d, size_t vsz) {
    size_t b = 2 * 3 * (size_t)d.Rx * padded_len(d.Kx) * vsz;
    if (d.flags & F_XSTAGE) b = xinv_stage_offset(3 * d.Rx, padded_len(d.Kx), vsz) + xinv_stage_bytes(d.Rx, d.nx, vsz / 2);
    return b;
}

// Cells per tile of the per-cell NEB kernels (rows of one plane, at least one row).
constexpr int kCellTile = 1024;

struct PlanItems {
    std::vector<WorkItem> x, y13, z, y2, yzc[kYzcListCount];
    std::vector<WorkItem> cell;   // per-cell tiles of ~kCellTile cells: rows of one plane
    size_t smem_x = 0, smem_xi = 0, smem_y13 = 0, smem_z = 0, smem_y2 = 0, smem_yzc = 0;
};

// Append the work items of simulation sid; vsz = bytes of one complex value.
inline void plan_items(const SimDesc& d, int sid, size_t vsz, PlanItems& P) {
    // x tiles: Rx consecutive rows of one plane (never crossing a plane)
    for (int z = 0; z < d.nz; ++z)
        for (int y0 = 0; y0 < d.ny; y0 += d.Rx) P.x.push_back({sid, z * d.ny + y0, std::min(d.Rx, d.ny - y0), 0});
    P.smem_x = std::max(P.smem_x, 2 * 3 * (size_t)d.Rx * padded_len(d.Kx) * vsz);
    P.smem_xi = std::max(P.smem_xi, plan_xinv_smem(d, vsz));
    const int rc = std::max(1, kCellTile / d.nx);
    for (int z = 0; z < d.nz; ++z)
        for (int y0 = 0; y0 < d.ny; y0 += rc) P.cell.push_back({sid, z * d.ny + y0, std::min(rc, d.ny - y0), 0});
    if (!(d.flags & F_DEMAG)) return;
    if (plan_uses_yzc(d)) {
        const int li = plan_yzc_list(d, vsz == 2 * sizeof(float));
        for (int b = 0; b < d.NBx; ++b) P.yzc[li].push_back({sid, 0, b, 0});
        P.smem_yzc = std::max(P.smem_yzc, 3 * (size_t)d.Py * d.Ty * vsz);
    } else if (d.Pz > 1) {
        if (d.Py > 1) {
            for (int z = 0; z < d.nz; ++z)
                for (int b = 0; b < d.NBx; ++b)
                    for (int c = 0; c < 3; ++c) P.y13.push_back({sid, z, b, c});
            P.smem_y13 = std::max(P.smem_y13, (size_t)d.Py * d.Ty * vsz);
        }
        for (int ky = 0; ky < d.Py; ++ky)
            for (int b = 0; b < d.NBx; ++b) P.z.push_back({sid, ky, b, 0});
        P.smem_z = std::max(P.smem_z, 3 * (size_t)d.Pz * d.Ty * vsz);
    } else if (d.Py > 1) {
        for (int b = 0; b < d.NBx; ++b) P.y2.push_back({sid, 0, b, -1});
        P.smem_y2 = std::max(P.smem_y2, 3 * (size_t)d.Py * d.Ty * vsz);
    }
}

}  // namespace mm

namespace mm {

// A planned simulation's tiles fit the kernels: Ty a power of two up to 32, at
// least one row per x tile, every pass's shared memory within one CTA's, and
// tuned CTA widths multiples of 32 up to maxthreads (the x and column kernels'
// launch bound).  vsz = bytes of one complex value.
inline bool plan_tuning_valid(const SimDesc& d, size_t vsz, const Tuning& t, int maxthreads) {
    if (d.Ty < 1 || d.Ty > 32 || (d.Ty & (d.Ty - 1)) || d.Rx < 1 || d.Rx > d.ny) return false;
    if (d.yzcocc && !(vsz == 8 && plan_uses_yzc(d) && d.nz <= kYzcOcc3MaxPlanes &&
                      d.yzcocc * ((size_t)3 * d.Py * d.Ty * vsz + 1024) <= 233472))
        return false;
    for (int th : {t.x_threads, t.col_threads})
        if (th != 0 && (th < 32 || th > maxthreads || th % 32)) return false;
    PlanItems P;
    SimDesc e = d;
    e.flags |= F_DEMAG;
    plan_items(e, 0, vsz, P);
    const size_t cap = 227 * 1024;
    return P.smem_x <= cap - 4096 && P.smem_xi <= cap - 4096 && P.smem_y13 <= cap && P.smem_y2 <= cap &&
           P.smem_z <= cap && P.smem_yzc <= cap;
}

// Candidates of one autotuning phase for the geometry of d0 (planned by the rule):
//   phase 0  kx block width Ty in {rule/2, rule, 2 rule} (at most the next power of
//            two above Kx) x, for FP32 cluster-pass films, both column group widths;
//   phase 1  with `fixed`'s Ty and groups: rows per x tile in {rule/2, rule, 2 rule}
//            x x-pass CTA width in {rule, 2 rule} x staged x-inverse rows off / on;
//   phase 2  with `fixed`'s other values: column-pass CTA width in {rule, 2 rule}
//            (meshes with column passes outside the cluster pass only).
// Every candidate passes plan_tuning_valid; the first is `fixed` itself.
inline std::vector<Tuning> plan_tuning_candidates(const SimDesc& d0, bool f32, int phase, const Tuning& fixed) {
    const size_t vsz = f32 ? 8 : 16;
    const int maxthreads = f32 ? 1024 : 512;
    std::vector<Tuning> out;
    auto add = [&](Tuning t) {
        SimDesc d = d0;
        plan_geometry(d, f32, t);
        if (!plan_tuning_valid(d, vsz, t, maxthreads)) return;
        for (const Tuning& u : out)
            if (u.Ty == t.Ty && u.Rx == t.Rx && u.x_threads == t.x_threads && u.col_threads == t.col_threads &&
                u.col_group == t.col_group && u.col_occ == t.col_occ && u.x_stage == t.x_stage)
                return;
        out.push_back(t);
    };
    add(fixed);
    SimDesc r = d0;
    plan_geometry(r, f32, fixed);
    if (phase == 0) {
        const int tymax = std::min(32, 1 << plan_ilog2(std::max(1, r.Kx)));
        const bool groups = f32 && plan_uses_yzc(r);
        const int g0 = plan_yzc_wide(plan_yzc_list(r, f32)) ? 2 : 1;
        for (int ty : {r.Ty / 2, r.Ty, 2 * r.Ty, r.Ty / 4})
            for (int occ : {0, 3, 4}) {
                if (ty < 1 || ty > tymax || (occ && !groups)) continue;
                for (int g : {g0, 3 - g0}) {
                    if (!groups && g != g0) continue;
                    Tuning t = fixed;
                    t.Ty = ty;
                    t.col_group = groups ? g : 0;
                    t.col_occ = occ;
                    add(t);
                }
            }
    } else if (phase == 1) {
        PlanItems P;
        SimDesc e = r;
        e.flags |= F_DEMAG;
        plan_items(e, 0, vsz, P);
        const int nt0 = plan_wide_threads(P.smem_x, maxthreads);
        for (int rx : {r.Rx / 2, r.Rx, 2 * r.Rx})
            for (int nt : {0, 2 * nt0})
                for (int st : {0, 1}) {
                    if (rx < 1) continue;
                    Tuning t = fixed;
                    t.Rx = rx;
                    t.x_threads = nt;
                    t.x_stage = st;
                    add(t);
                }
    } else if (phase == 2) {
        PlanItems P;
        SimDesc e = r;
        e.flags |= F_DEMAG;
        plan_items(e, 0, vsz, P);
        const size_t sc = std::max(P.smem_y13, std::max(P.smem_z, P.smem_y2));
        if (sc > 0) {
            Tuning t = fixed;
            t.col_threads = 2 * plan_wide_threads(sc, maxthreads);
            add(t);
        }
    }
    return out;
}

}  // namespace mm
