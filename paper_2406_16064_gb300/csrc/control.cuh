// Step control, projection and NEB kernels.
//
//  k_after_stage1  per simulation: max|dm/dt| of stage 1, relaxation stop
//                  test (max|dm/dt| < max_dmdt), initial step
//                  h0 = min(1e-12 s, 0.01 / max|dm/dt|).
//  k_controller    per simulation: accept when err = max|h sum e_j k_j| / rtol
//                  <= 1, h <- h clamp(0.9 err^-1/5, 0.2, 5), clip to t_end
//                  (adaptive Dormand-Prince, Sec. "LLG equation").  NEB chain
//                  members share err (max over the chain) and so h.
//  k_project       m <- y5 / |y5| for accepted simulations (the projection onto
//                  |m| = 1 after every successful step), norm in FP64.
//  k_neb_tangent / k_neb_force
//                  geodesic NEB (Sec. "Miscellaneous"): energy-weighted upwind
//                  tangent projected onto the tangent planes, geodesic image
//                  distances, force H - (H.tau) tau + k (L+ - L-) tau and the
//                  precession-free LL torque -alpha g~ m x (m x F).
#pragma once
#include "passes.cuh"

namespace mm {

__device__ __forceinline__ unsigned long long group_max(const SimDesc* desc, const SimState* st, int s,
                                                        bool err) {
    unsigned long long b = err ? st[s].err_bits : st[s].maxk_bits;
    const int gb = desc[s].group_begin, ge = desc[s].group_end;
    if (gb >= 0) {
        for (int i = gb; i < ge; ++i) {
            const unsigned long long v = err ? st[i].err_bits : st[i].maxk_bits;
            b = v > b ? v : b;
        }
    }
    return b;
}

static __global__ void k_after_stage1(const SimDesc* desc, SimState* st, int nsims) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsims) return;
    SimState& S = st[s];
    if (S.status != 0) return;
    const double mk = sqrt(bits_to_double(group_max(desc, st, s, false)));   // max |dm/dt|^2 -> max |dm/dt|
    S.maxk = mk;
    S.err_bits = 0ull;
    if (!(mk == mk) || isinf(mk)) { S.status = -4; return; }
    if (S.max_dmdt > 0.0 && mk < S.max_dmdt) { S.status = 2; return; }
    if (S.h <= 0.0) {
        double h = mk > 0.0 ? fmin(1e-12, 0.01 / mk) : 1e-12;
        if (S.t_end > 0.0) h = fmin(h, S.t_end - S.t);
        S.h = h;
    }
}

static __global__ void k_controller(const SimDesc* desc, SimState* st, int nsims) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsims) return;
    SimState& S = st[s];
    S.maxk_bits = 0ull;
    if (S.status != 0) { S.accepted = 0; return; }
    const double err = bits_to_double(group_max(desc, st, s, true)) / S.rtol;
    S.err = err;
    if (!(err == err) || isinf(err)) { S.status = -4; S.accepted = 0; return; }
    const int acc = err <= 1.0;
    double h = S.h;
    if (acc) { S.t += h; S.n_acc += 1; } else { S.n_rej += 1; }
    S.accepted = acc;
    const double f = err == 0.0 ? 5.0 : fmin(5.0, fmax(0.2, 0.9 * pow(err, -0.2)));
    h *= f;
    if (S.t_end > 0.0) {
        h = fmin(h, S.t_end - S.t);
        if (S.t_end - S.t <= 1e-12 * S.t_end) S.status = 1;
    }
    S.h = h;
    if (S.status == 0 && !(h > 1e-24)) S.status = -5;
}

// 1/sqrt(s) for the projection: the sum of squares s is formed in FP64; an
// FP32 rsqrt seed (relative error ~1e-7) is refined by Newton-Raphson steps
// y <- y (3 - s y^2) / 2 in FP64, each squaring the relative error (one step
// for FP32 states, two for FP64).  Returns 1 for s = 0.
template <typename T>
__device__ __forceinline__ double inv_norm(double s) {
    if (!(s > 0.0)) return 1.0;
    double y = (double)rsqrtf((float)s);
    y = y * (1.5 - 0.5 * s * y * y);
    if (sizeof(T) == 8) y = y * (1.5 - 0.5 * s * y * y);
    return y;
}

// m <- y / |y| for one cell.  FP64 states: sum of squares and Newton-refined
// rsqrt in FP64.  FP32 states: the same accuracy from FP32 operations in
// float-float arithmetic (error-free products and sums, one Newton step on
// the unevaluated sum hi + lo), since FP64 instructions would bound the
// kernel on GB300: 1/|y| comes out to ~1e-13 relative and each component is
// rounded once, as the FP64 form rounds (T)(y_c / |y|).
__device__ __forceinline__ void project_cell(const double (&y)[3], double (&m)[3]) {
    const double inv = inv_norm<double>(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
#pragma unroll
    for (int c = 0; c < 3; ++c) m[c] = y[c] * inv;
}

__device__ __forceinline__ void project_cell(const float (&y)[3], float (&m)[3]) {
    float p0, e0, p1, e1, p2, e2, s, t1, t2;
    two_prod(y[0], y[0], p0, e0);
    two_prod(y[1], y[1], p1, e1);
    two_prod(y[2], y[2], p2, e2);
    two_sum(p0, p1, s, t1);
    two_sum(s, p2, s, t2);
    const float lo = __fadd_rn(__fadd_rn(__fadd_rn(e0, e1), __fadd_rn(e2, t1)), t2);   // |y|^2 = s + lo
    if (!(s > 0.f)) {                      // zero (or non-finite) vector: unchanged, as the FP64 form
#pragma unroll
        for (int c = 0; c < 3; ++c) m[c] = y[c];
        return;
    }
    const float r0 = rsqrtf(s);
    // q = 1 - |y|^2 r0^2 to ~eps^2: r0^2 = a + ae and s a = b + be exactly, 1 - b exact (b ~ 1)
    float a, ae, b, be;
    two_prod(r0, r0, a, ae);
    two_prod(s, a, b, be);
    const float q = __fsub_rn(__fsub_rn(__fsub_rn(1.f, b), be), __fmaf_rn(s, ae, __fmul_rn(lo, a)));
    const float rl = __fmul_rn(__fmul_rn(0.5f, r0), q);   // 1/|y| = r0 + rl (one Newton step)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float pc, ec;
        two_prod(y[c], r0, pc, ec);
        m[c] = __fadd_rn(pc, __fmaf_rn(y[c], rl, ec));
    }
}

template <typename T>
__global__ void __launch_bounds__(MM_THREADS) k_project(const SimDesc* __restrict__ desc, const SimState* st,
                                                        const WorkItem* __restrict__ items, T* m, const T* y) {
    const WorkItem w = items[blockIdx.x];
    const SimState& S = st[w.sim];
    if (!S.accepted) return;                       // rejected, or not running
    const SimDesc& d = desc[w.sim];
    if (d.group_begin >= 0 && (d.neb_index == 0 || d.neb_index == d.group_end - d.group_begin - 1))
        return;                                    // NEB end images stay bit-fixed
    const long long N = d.ncells;
    const long long c0 = d.off + (long long)w.a * d.nx;
    const int cnt = w.b * d.nx;
    // four cells per thread per pass: all twelve loads in flight before the stores
    for (int b0 = threadIdx.x; b0 < cnt; b0 += 4 * blockDim.x) {
        T v[4][3];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int id = b0 + u * blockDim.x;
            const long long o = c0 + (id < cnt ? id : 0);
#pragma unroll
            for (int c = 0; c < 3; ++c) v[u][c] = y[o + c * N];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int id = b0 + u * blockDim.x;
            if (id >= cnt) continue;
            const long long o = c0 + id;
            T r[3];
            project_cell(v[u], r);
#pragma unroll
            for (int c = 0; c < 3; ++c) m[o + c * N] = r[c];
        }
    }
}

// ------------------------------------------------------------------- NEB
template <typename T>
struct NebParams {
    const SimDesc* __restrict__ desc;
    SimState* state;
    const WorkItem* __restrict__ items;
    const T* ys;          // stage state of every image
    const T* heff;        // effective field of every image
    T* tau;               // raw projected tangent
    T* kout;              // k_s
    const T* errp;
    const T* __restrict__ Ms;
    int stage;
    double e7;
};

static __global__ void k_neb_reset(SimState* st, int nsims) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsims) return;
    for (int i = 0; i < 8; ++i) st[s].E[i] = 0.0;
    for (int i = 0; i < 4; ++i) st[s].neb[i] = 0.0;
}

__device__ __forceinline__ double total_energy(const SimState& S) {
    return S.E[0] + S.E[1] + S.E[2] + S.E[3] + S.E[4] + S.E[5];
}

// Block sum of per-thread compensated sums: warp sums in the context
// precision (float-float for FP32), the cross-warp sum in FP64.  Result in
// thread 0.
template <typename T>
__device__ __forceinline__ double block_csum(CSum<T> v, double* red) {
    v.warp_reduce();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v.value();
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += red[i];
    }
    return r;
}

// Three block sums at once (one pair of barriers): results in r[0..2] of thread 0.
template <typename T>
__device__ __forceinline__ void block_csum3(CSum<T> a, CSum<T> b, CSum<T> c, double* red, double (&r)[3]) {
    a.warp_reduce();
    b.warp_reduce();
    c.warp_reduce();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    __syncthreads();
    if (lane == 0) {
        red[wid] = a.value();
        red[nw + wid] = b.value();
        red[2 * nw + wid] = c.value();
    }
    __syncthreads();
    r[0] = r[1] = r[2] = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < nw; ++i) {
            r[0] += red[i];
            r[1] += red[nw + i];
            r[2] += red[2 * nw + i];
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(MM_THREADS) k_neb_tangent(NebParams<T> p) {
    __shared__ double red[3 * MM_THREADS / 32];
    __shared__ T wsh[2];
    const WorkItem w = p.items[blockIdx.x];
    SimState* st = p.state;
    if (st[w.sim].status != 0) return;
    const SimDesc& d = p.desc[w.sim];
    const int i = d.neb_index, n = d.group_end - d.group_begin;
    const int N = d.ncells;
    const bool free_img = i > 0 && i < n - 1;
    const bool has_next = i < n - 1;
    if (threadIdx.x == 0) {
        // tau = wp * tau+ + wm * tau- (energy-weighted upwind tangent), in FP64 once per CTA
        double wp = 0.0, wm = 0.0;
        if (free_img) {
            const double Ep = total_energy(st[w.sim + 1]), E0 = total_energy(st[w.sim]),
                         Em = total_energy(st[w.sim - 1]);
            if (Ep > E0 && E0 > Em) { wp = 1.0; wm = 0.0; }
            else if (Ep < E0 && E0 < Em) { wp = 0.0; wm = 1.0; }
            else {
                const double dmax = fmax(fabs(Ep - E0), fabs(Em - E0));
                const double dmin = fmin(fabs(Ep - E0), fabs(Em - E0));
                if (Ep > Em) { wp = dmax; wm = dmin; } else { wp = dmin; wm = dmax; }
            }
            // only the direction of tau matters (it is normalised per image): scale the
            // weights to <= 1 so the per-cell products stay in range in FP32
            const double wn = fmax(wp, wm);
            if (wn > 0.0) { wp /= wn; wm /= wn; }
        }
        wsh[0] = (T)wp;
        wsh[1] = (T)wm;
    }
    __syncthreads();
    const long long off = d.off;
    const long long offn = has_next ? p.desc[w.sim + 1].off : off;
    const long long offp = free_img ? p.desc[w.sim - 1].off : off;
    // per-cell geometry in the context precision, compensated per-thread sums, FP64 across threads
    CSum<T> t2, ht, th2;
    const T wpt = wsh[0], wmt = wsh[1];
    const long long c0 = (long long)w.a * d.nx;
    const int cnt = w.b * d.nx;
    for (int id = threadIdx.x; id < cnt; id += blockDim.x) {
        const long long cell = c0 + id;
        T m[3], mn[3], mp[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            m[c] = p.ys[off + c * (long long)N + cell];
            mn[c] = p.ys[offn + c * (long long)N + cell];
            mp[c] = p.ys[offp + c * (long long)N + cell];
        }
        if (has_next) {
            const T cx = m[1] * mn[2] - m[2] * mn[1], cy = m[2] * mn[0] - m[0] * mn[2],
                    cz = m[0] * mn[1] - m[1] * mn[0];
            const T th = atan2(sqrt(cx * cx + cy * cy + cz * cz), m[0] * mn[0] + m[1] * mn[1] + m[2] * mn[2]);
            th2.add(th * th);
        }
        if (free_img) {
            T t[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) t[c] = wpt * (mn[c] - m[c]) + wmt * (m[c] - mp[c]);
            const T tm = t[0] * m[0] + t[1] * m[1] + t[2] * m[2];
#pragma unroll
            for (int c = 0; c < 3; ++c) t[c] -= tm * m[c];
            T tt = 0, htc = 0;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                p.tau[off + c * (long long)N + cell] = t[c];
                tt += t[c] * t[c];
                htc += p.heff[off + c * (long long)N + cell] * t[c];
            }
            t2.add(tt);
            ht.add(htc);
        }
    }
    double sums[3];
    block_csum3(t2, ht, th2, red, sums);
    if (threadIdx.x == 0) {
        atomicAdd(&st[w.sim].neb[0], sums[0]);
        atomicAdd(&st[w.sim].neb[1], sums[1]);
        atomicAdd(&st[w.sim].neb[2], sums[2]);
    }
}

template <typename T>
__global__ void __launch_bounds__(MM_THREADS) k_neb_force(NebParams<T> p) {
    __shared__ unsigned long long red[MM_THREADS / 32];
    __shared__ T fsh[3];
    const WorkItem w = p.items[blockIdx.x];
    SimState* st = p.state;
    if (st[w.sim].status != 0) return;
    const SimDesc& d = p.desc[w.sim];
    const int i = d.neb_index, n = d.group_end - d.group_begin;
    const int N = d.ncells;
    const bool free_img = i > 0 && i < n - 1;
    const bool msarr = (d.flags & F_MSARR) != 0;
    if (threadIdx.x == 0) {
        // 1/|tau|, H.tau/|tau| and the spring term k (L+ - L-) in FP64 once per CTA
        double inv_t = 0.0, Ht = 0.0, spring = 0.0;
        if (free_img) {
            const double t2 = st[w.sim].neb[0];
            inv_t = t2 > 0.0 ? 1.0 / sqrt(t2) : 0.0;
            Ht = st[w.sim].neb[1] * inv_t;
            spring = d.k_spring * (sqrt(st[w.sim].neb[2]) - sqrt(st[w.sim - 1].neb[2]));
        }
        fsh[0] = (T)inv_t;
        fsh[1] = (T)Ht;
        fsh[2] = (T)spring;
    }
    __syncthreads();
    const long long off = d.off;
    const long long c0 = (long long)w.a * d.nx;
    const int cnt = w.b * d.nx;
    const T inv_tt = fsh[0], Htt = fsh[1], springt = fsh[2], agtt = coef<T>(d).agt;
    const T e7 = (T)p.e7;
    unsigned long long vmax = 0ull;
    for (int id = threadIdx.x; id < cnt; id += blockDim.x) {
        const long long cell = c0 + id;
        const bool mag = !msarr || p.Ms[d.ms_off + cell] > (T)0;
        T k[3] = {(T)0, (T)0, (T)0};
        if (free_img && mag) {
            T m[3], F[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                m[c] = p.ys[off + c * (long long)N + cell];
                const T tc = p.tau[off + c * (long long)N + cell] * inv_tt;
                F[c] = p.heff[off + c * (long long)N + cell] - Htt * tc + springt * tc;
            }
            const T c0x = m[1] * F[2] - m[2] * F[1], c0y = m[2] * F[0] - m[0] * F[2],
                    c0z = m[0] * F[1] - m[1] * F[0];
            k[0] = -agtt * (m[1] * c0z - m[2] * c0y);
            k[1] = -agtt * (m[2] * c0x - m[0] * c0z);
            k[2] = -agtt * (m[0] * c0y - m[1] * c0x);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) p.kout[off + c * (long long)N + cell] = k[c];
        if (p.stage == 1) {
            vmax = umax64(vmax, obits(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]));      // squared norm
        } else if (p.stage == 7) {
            // e_7 k_7 added to the prologue's partial sum in one FMA; h after the max
#pragma unroll
            for (int c = 0; c < 3; ++c)
                vmax = umax64(vmax, obits(fabs(fma(e7, k[c], p.errp[off + c * (long long)N + cell]))));
        }
    }
    if (p.stage == 1 || p.stage == 7) {
        const unsigned long long r = block_max_u64(vmax, red);
        if (threadIdx.x == 0) {
            const double v = obits_to_double<T>(r);
            const double vs = p.stage == 7 ? fabs(st[w.sim].h * v) : v;
            atomicMax(p.stage == 1 ? &st[w.sim].maxk_bits : &st[w.sim].err_bits,
                      (unsigned long long)__double_as_longlong(vs));
        }
    }
}

// A wait on a device flag that nothing sets, bounded by `spins` polls;
// reports MM_ETIMEOUT through *status instead of hanging.
static __global__ void k_bounded_wait(volatile int* flag, long long spins, int* status) {
    long long i = 0;
    while (*flag == 0 && i < spins) ++i;
    *status = (*flag == 0) ? -6 : 0;
}

}  // namespace mm
