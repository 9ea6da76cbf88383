// Kernel sequencing of the right-hand side and of one RK45 attempt.
#pragma once
#include <cstring>

#include "control.cuh"
#include "engine.cuh"

namespace mm {

// C: compute type of the transforms (float, double or dd); the state pointers
// of PassParams<C> are of its storage type StoreT<C>.
template <typename C>
static PassParams<C> base_params(const Launch& L) {
    using S = StoreT<C>;
    PassParams<C> p;
    memset(&p, 0, sizeof(p));
    p.desc = L.desc;
    p.state = L.state;
    p.spec = reinterpret_cast<V2<C>*>(L.spec);
    p.tensor = reinterpret_cast<const C*>(L.tensor);
    p.Ms = reinterpret_cast<const S*>(L.Ms);
    p.cellp = reinterpret_cast<const S*>(L.cellp);
    p.tw = reinterpret_cast<const V2<C>*>(L.tw);
    for (int j = 0; j < 7; ++j) p.e[j] = dp_e(j);
    return p;
}

// Threads of an x- or column-pass CTA: the tuned width when the batch has one
// (Launch::x_threads / col_threads), else the fixed rule (plan_wide_threads: 32
// warps FP32, 16 FP64 per SM, the register budget of those kernels' launch bounds).
template <typename T>
static int wide_threads(size_t smem, int tuned = 0) {
    if (tuned >= 32 && tuned <= MM_XTHREADS_MAX<T> && tuned % 32 == 0) return tuned;
    return plan_wide_threads(smem, MM_XTHREADS_MAX<T>);
}

// The cluster kernel for nz planes (2..8), the column group width and the CTAs
// per SM it is built for (occ 3 or 4: FP32 up to kYzcOcc3MaxPlanes planes).
template <typename T>
static void (*yzc_kernel(int nz, bool wide, int occ = 2))(PassParams<T>) {
    if (occ == 3 && sizeof(T) == 4 && nz <= kYzcOcc3MaxPlanes) {
        switch (nz) {
            case 2: return wide ? k_yzc<T, 2, true, 3> : k_yzc<T, 2, false, 3>;
            case 3: return wide ? k_yzc<T, 3, true, 3> : k_yzc<T, 3, false, 3>;
            default: return wide ? k_yzc<T, 4, true, 3> : k_yzc<T, 4, false, 3>;
        }
    }
    if (occ == 4 && sizeof(T) == 4 && nz <= kYzcOcc3MaxPlanes) {
        switch (nz) {
            case 2: return wide ? k_yzc<T, 2, true, 4> : k_yzc<T, 2, false, 4>;
            case 3: return wide ? k_yzc<T, 3, true, 4> : k_yzc<T, 3, false, 4>;
            default: return wide ? k_yzc<T, 4, true, 4> : k_yzc<T, 4, false, 4>;
        }
    }
    switch (nz) {
        case 2: return wide ? k_yzc<T, 2, true> : k_yzc<T, 2, false>;
        case 3: return wide ? k_yzc<T, 3, true> : k_yzc<T, 3, false>;
        case 4: return wide ? k_yzc<T, 4, true> : k_yzc<T, 4, false>;
        case 5: return wide ? k_yzc<T, 5, true> : k_yzc<T, 5, false>;
        case 6: return wide ? k_yzc<T, 6, true> : k_yzc<T, 6, false>;
        case 7: return wide ? k_yzc<T, 7, true> : k_yzc<T, 7, false>;
        default: return wide ? k_yzc<T, 8, true> : k_yzc<T, 8, false>;
    }
}

template <typename T>
static void issue_passes(const Launch& L, PassParams<T> p, const StoreT<T>* ys, bool include_xinv = true) {
    if (L.x.count == 0) return;
    cudaStream_t s = L.stream;
    ProfileHook* hk = L.hook;
    p.items = L.x.dev;
    const int ntx = wide_threads<T>(L.smem_x, L.x_threads), ntxi = wide_threads<T>(L.smem_xi + 2048, L.x_threads);
    switch ((p.mode == MODE_RK || p.mode == MODE_NEB) ? p.stage : 0) {
        case 2: k_xfwd<T, 2><<<L.x.count, ntx, L.smem_x, s>>>(p); break;
        case 3: k_xfwd<T, 3><<<L.x.count, ntx, L.smem_x, s>>>(p); break;
        case 4: k_xfwd<T, 4><<<L.x.count, ntx, L.smem_x, s>>>(p); break;
        case 5: k_xfwd<T, 5><<<L.x.count, ntx, L.smem_x, s>>>(p); break;
        case 6: k_xfwd<T, 6><<<L.x.count, ntx, L.smem_x, s>>>(p); break;
        case 7: k_xfwd<T, 7><<<L.x.count, ntx, L.smem_x, s>>>(p); break;
        default: k_xfwd<T, 0><<<L.x.count, ntx, L.smem_x, s>>>(p); break;
    }
    if (hk) hk->mark(KIND_XFWD);
    long long n = 1;
    if (L.y13.count) {
        p.items = L.y13.dev;
        k_ycol<T, 0><<<L.y13.count, wide_threads<T>(L.smem_y13, L.col_threads), L.smem_y13, s>>>(p);
        if (hk) hk->mark(KIND_YFWD);
        ++n;
    }
    if (L.z.count) {
        p.items = L.z.dev;
        k_zcol<T><<<L.z.count, wide_threads<T>(L.smem_z, L.col_threads), L.smem_z, s>>>(p);
        if (hk) hk->mark(KIND_ZCOL);
        ++n;
    }
    if (L.y13.count) {
        p.items = L.y13.dev;
        k_ycol<T, 1><<<L.y13.count, wide_threads<T>(L.smem_y13, L.col_threads), L.smem_y13, s>>>(p);
        if (hk) hk->mark(KIND_YINV);
        ++n;
    }
    for (int li = 0; li < kYzcListCount; ++li) {
        if (!L.yzc[li].count) continue;
        const int nz = li % kYzcLists;
        const bool wide = ((li / kYzcLists) & 1) != 0;
        const int occ = 2 + li / (2 * kYzcLists);
        p.items = L.yzc[li].dev;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(L.yzc[li].count * nz), 1, 1);
        cfg.blockDim = dim3(MM_THREADS, 1, 1);
        cfg.dynamicSmemBytes = L.smem_yzc;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = nz;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        // one instantiation per plane count; wide: 32-point column groups
        cudaLaunchKernelEx(&cfg, yzc_kernel<T>(nz, wide, occ), p);
        if (hk) hk->mark(KIND_YZC);
        ++n;
    }
    if (L.y2.count) {
        p.items = L.y2.dev;
        k_ycol<T, 2><<<L.y2.count, wide_threads<T>(L.smem_y2, L.col_threads), L.smem_y2, s>>>(p);
        if (hk) hk->mark(KIND_YFUSED);
        ++n;
    }
    if (include_xinv) {
        p.items = L.x.dev;
        const bool en = p.mode == MODE_ENERGY || p.mode == MODE_NEB;
        if (L.ext) {
            if (en) k_xinv<T, true, true><<<L.x.count, ntxi, L.smem_xi, s>>>(p, ys);
            else k_xinv<T, false, true><<<L.x.count, ntxi, L.smem_xi, s>>>(p, ys);
        } else {
            if (en) k_xinv<T, true, false><<<L.x.count, ntxi, L.smem_xi, s>>>(p, ys);
            else k_xinv<T, false, false><<<L.x.count, ntxi, L.smem_xi, s>>>(p, ys);
        }
        if (hk) hk->mark(KIND_XINV);
        ++n;
    }
    if (L.launches) *L.launches += n;
}

template <typename S, typename C>
void engine_rhs_c(const Launch& L, int mode, const S* m, S* dmdt, S* heff, long long off_adjust) {
    PassParams<C> p = base_params<C>(L);
    p.mode = mode;
    p.m = m;
    p.kout = dmdt;
    p.heff = heff;
    p.off_adjust = off_adjust;
    issue_passes<C>(L, p, m);
}

static inline int blocks_for(int n) { return (n + 127) / 128; }

template <typename S, typename C>
void engine_attempt_c(const Launch& L, const RkBuffers& B) {
    cudaStream_t s = L.stream;
    for (int st = 1; st <= 7; ++st) {
        PassParams<C> p = base_params<C>(L);
        p.mode = MODE_RK;
        p.stage = st;
        p.nk = st - 1;
        p.write_y = st > 1;
        for (int j = 0; j < 6; ++j) p.a[j] = dp_a(st, j);
        p.m = reinterpret_cast<const S*>(B.m);
        p.ybuf = reinterpret_cast<S*>(B.ybuf);
        p.kvec = reinterpret_cast<S* const*>(B.kvec_dev);
        p.kout = reinterpret_cast<S*>(B.kvec[st - 1]);
        p.errp = reinterpret_cast<S*>(B.errp);
        const S* ys = st == 1 ? reinterpret_cast<const S*>(B.m) : reinterpret_cast<const S*>(B.ybuf);
        issue_passes<C>(L, p, ys);
        if (st == 1) {
            k_after_stage1<<<blocks_for(L.nsims), 128, 0, s>>>(L.desc, L.state, L.nsims);
            if (L.hook) L.hook->mark(KIND_CONTROL);
            if (L.launches) *L.launches += 1;
        }
    }
    k_controller<<<blocks_for(L.nsims), 128, 0, s>>>(L.desc, L.state, L.nsims);
    if (L.hook) L.hook->mark(KIND_CONTROL);
    k_project<S><<<L.x.count, MM_THREADS, 0, s>>>(L.desc, L.state, L.x.dev, reinterpret_cast<S*>(B.m),
                                                  reinterpret_cast<const S*>(B.ybuf));
    if (L.hook) L.hook->mark(KIND_PROJECT);
    if (L.launches) *L.launches += 2;
}

template <typename S, typename C>
void engine_neb_attempt_c(const Launch& L, const RkBuffers& B) {
    cudaStream_t s = L.stream;
    for (int st = 1; st <= 7; ++st) {
        k_neb_reset<<<blocks_for(L.nsims), 128, 0, s>>>(L.state, L.nsims);
        if (L.hook) L.hook->mark(KIND_CONTROL);
        PassParams<C> p = base_params<C>(L);
        p.mode = MODE_NEB;
        p.stage = st;
        p.nk = st - 1;
        p.write_y = st > 1;
        for (int j = 0; j < 6; ++j) p.a[j] = dp_a(st, j);
        p.m = reinterpret_cast<const S*>(B.m);
        p.ybuf = reinterpret_cast<S*>(B.ybuf);
        p.kvec = reinterpret_cast<S* const*>(B.kvec_dev);
        p.kout = nullptr;
        p.heff = reinterpret_cast<S*>(B.heff);
        p.errp = reinterpret_cast<S*>(B.errp);
        const S* ys = st == 1 ? reinterpret_cast<const S*>(B.m) : reinterpret_cast<const S*>(B.ybuf);
        issue_passes<C>(L, p, ys);
        NebParams<S> q;
        q.desc = L.desc;
        q.state = L.state;
        q.items = L.cell.dev;
        q.ys = ys;
        q.heff = reinterpret_cast<const S*>(B.heff);
        q.tau = reinterpret_cast<S*>(B.tau);
        q.kout = reinterpret_cast<S*>(B.kvec[st - 1]);
        q.errp = reinterpret_cast<const S*>(B.errp);
        q.Ms = reinterpret_cast<const S*>(L.Ms);
        q.stage = st;
        q.e7 = dp_e(6);
        k_neb_tangent<S><<<L.cell.count, MM_THREADS, 0, s>>>(q);
        k_neb_force<S><<<L.cell.count, MM_THREADS, 0, s>>>(q);
        if (L.hook) L.hook->mark(KIND_NEB);
        if (L.launches) *L.launches += 3;
        if (st == 1) {
            k_after_stage1<<<blocks_for(L.nsims), 128, 0, s>>>(L.desc, L.state, L.nsims);
            if (L.hook) L.hook->mark(KIND_CONTROL);
            if (L.launches) *L.launches += 1;
        }
    }
    k_controller<<<blocks_for(L.nsims), 128, 0, s>>>(L.desc, L.state, L.nsims);
    if (L.hook) L.hook->mark(KIND_CONTROL);
    k_project<S><<<L.x.count, MM_THREADS, 0, s>>>(L.desc, L.state, L.x.dev, reinterpret_cast<S*>(B.m),
                                                  reinterpret_cast<const S*>(B.ybuf));
    if (L.hook) L.hook->mark(KIND_PROJECT);
    if (L.launches) *L.launches += 2;
}

// The entry points, per storage type.  An FP64 launch with Launch::dd set runs its
// transforms in double-float (engine_dd.cu); everything else in the storage type.
template <typename S>
void engine_rhs(const Launch& L, int mode, const S* m, S* dmdt, S* heff, long long off_adjust) {
    if constexpr (sizeof(S) == 8) {
        if (L.dd) { engine_rhs_dd(L, mode, m, dmdt, heff, off_adjust); return; }
    }
    engine_rhs_c<S, S>(L, mode, m, dmdt, heff, off_adjust);
}

template <typename S>
void engine_attempt(const Launch& L, const RkBuffers& B) {
    if constexpr (sizeof(S) == 8) {
        if (L.dd) { engine_attempt_dd(L, B); return; }
    }
    engine_attempt_c<S, S>(L, B);
}

template <typename S>
void engine_neb_attempt(const Launch& L, const RkBuffers& B) {
    if constexpr (sizeof(S) == 8) {
        if (L.dd) { engine_neb_attempt_dd(L, B); return; }
    }
    engine_neb_attempt_c<S, S>(L, B);
}

template <typename T>
static void set_attrs() {
    const int mx = 227 * 1024;
    cudaFuncSetAttribute(k_xfwd<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_xfwd<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_xfwd<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_xfwd<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_xfwd<T, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_xfwd<T, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_xfwd<T, 7>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_xinv<T, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx - 4096);
    cudaFuncSetAttribute(k_xinv<T, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx - 4096);
    cudaFuncSetAttribute(k_xinv<T, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx - 4096);
    cudaFuncSetAttribute(k_xinv<T, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx - 4096);
    cudaFuncSetAttribute(k_ycol<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_ycol<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_ycol<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_zcol<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    for (int nz = 2; nz <= 8; ++nz)
        for (int v = 0; v < 6; ++v)
            cudaFuncSetAttribute(yzc_kernel<T>(nz, (v & 1) != 0, 2 + v / 2),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
}

}  // namespace mm
