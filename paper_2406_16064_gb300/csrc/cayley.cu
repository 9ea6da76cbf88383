// Fixed-step classical Runge-Kutta (RK4) for every simulation of a context,
// with projection onto |m| = 1 after the step, or on the Cayley-transform
// variable (Sec. "Cayley transform").  With dm/dt = f x m,
// f = gamma (H + alpha m x H) / (1 + alpha^2) (precession off: only the alpha
// term), m(t) = Q(omega) m_n with Q = (I - Omega/2)^-1 (I + Omega/2),
// Omega = skew[omega], and d omega/dt = f - (omega x f)/2 + (omega . f) omega/4.
// omega restarts from 0 at every step; m_{n+1} = Q(omega_{n+1}) m_n.
//
// One step = four effective-field evaluations (the right-hand-side passes)
// and these kernels, captured as one CUDA graph per call:
//   k_c4_stage  stage state: m_n + c h k_prev (projection), or
//               Q(c h k_prev) m_n (Cayley, closed form per cell)
//   k_c4_omega  Cayley: k_s = d omega/dt at omega = c h k_prev from the
//               stage's m and H (projection: k_s is the right-hand side the
//               passes write directly)
//   k_c4_final  m_{n+1} from h/6 (k1 + 2 k2 + 2 k3 + k4): Q(.) m_n, or
//               m_n + (.) projected onto |m| = 1; cells with Ms = 0 stay
//   k_c4_time   t += h
#include "cayley.h"
#include "control.cuh"

namespace mm {

template <typename T>
__device__ __forceinline__ void cx3(const T (&a)[3], const T (&b)[3], T (&c)[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// Q(w) m, Q = (I - W/2)^-1 (I + W/2): b = m + w x m / 2, then
// (I - W/2)^-1 b = (b + w x b / 2 + (w.b) w / 4) / (1 + |w|^2 / 4)
template <typename T>
__device__ __forceinline__ void cayley_map(const T (&w)[3], const T (&m)[3], T (&out)[3]) {
    T wm[3], b[3], wb[3];
    cx3(w, m, wm);
#pragma unroll
    for (int c = 0; c < 3; ++c) b[c] = m[c] + (T)0.5 * wm[c];
    cx3(w, b, wb);
    const T wdb = w[0] * b[0] + w[1] * b[1] + w[2] * b[2];
    const T inv = (T)1 / ((T)1 + (T)0.25 * (w[0] * w[0] + w[1] * w[1] + w[2] * w[2]));
#pragma unroll
    for (int c = 0; c < 3; ++c) out[c] = (b[c] + (T)0.5 * wb[c] + (T)0.25 * wdb * w[c]) * inv;
}

template <typename T, bool CAY>
__global__ void __launch_bounds__(MM_THREADS) k_c4_stage(const SimDesc* __restrict__ desc,
                                                         const WorkItem* __restrict__ items, const T* m,
                                                         const T* kprev, double ch, T* ys) {
    const WorkItem w = items[blockIdx.x];
    const SimDesc& d = desc[w.sim];
    const long long N = d.ncells;
    const long long c0 = d.off + (long long)w.a * d.nx;
    const int cnt = w.b * d.nx;
    const T c = (T)ch;
    for (int id = threadIdx.x; id < cnt; id += blockDim.x) {
        const long long o = c0 + id;
        T mv[3], wv[3], out[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) { mv[q] = m[o + q * N]; wv[q] = c * kprev[o + q * N]; }
        if (CAY) {
            cayley_map(wv, mv, out);
        } else {
#pragma unroll
            for (int q = 0; q < 3; ++q) out[q] = mv[q] + wv[q];
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) ys[o + q * N] = out[q];
    }
}

template <typename T>
__global__ void __launch_bounds__(MM_THREADS) k_c4_omega(const SimDesc* __restrict__ desc,
                                                         const WorkItem* __restrict__ items, const T* ms,
                                                         const T* H, const T* kprev, double ch, T* kout,
                                                         const T* __restrict__ Ms) {
    const WorkItem w = items[blockIdx.x];
    const SimDesc& d = desc[w.sim];
    const long long N = d.ncells;
    const long long c0 = d.off + (long long)w.a * d.nx;
    const int cnt = w.b * d.nx;
    const bool msarr = (d.flags & F_MSARR) != 0;
    const T* __restrict__ msp = msarr ? Ms + d.ms_off + (long long)w.a * d.nx : nullptr;
    const Coef<T>& cf = coef<T>(d);
    const bool prec = (d.flags & F_PREC) != 0;
    const T c = (T)ch, gt = cf.gt, agt = cf.agt;
    for (int id = threadIdx.x; id < cnt; id += blockDim.x) {
        const long long o = c0 + id;
        T mv[3], Hv[3], mxH[3], f[3], wv[3] = {(T)0, (T)0, (T)0}, wxf[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            mv[q] = ms[o + q * N];
            Hv[q] = H[o + q * N];
            if (kprev) wv[q] = c * kprev[o + q * N];
        }
        cx3(mv, Hv, mxH);
        const bool has = !msarr || msp[id] > (T)0;   // f = 0 where there is no magnetisation
#pragma unroll
        for (int q = 0; q < 3; ++q) f[q] = has ? agt * mxH[q] + (prec ? gt * Hv[q] : (T)0) : (T)0;
        cx3(wv, f, wxf);
        const T wdf = wv[0] * f[0] + wv[1] * f[1] + wv[2] * f[2];
#pragma unroll
        for (int q = 0; q < 3; ++q) kout[o + q * N] = f[q] - (T)0.5 * wxf[q] + (T)0.25 * wdf * wv[q];
    }
}

template <typename T, bool CAY>
__global__ void __launch_bounds__(MM_THREADS) k_c4_final(const SimDesc* __restrict__ desc,
                                                         const WorkItem* __restrict__ items, T* m, const T* k1,
                                                         const T* k2, const T* k3, const T* k4, double h6,
                                                         const T* __restrict__ Ms) {
    const WorkItem w = items[blockIdx.x];
    const SimDesc& d = desc[w.sim];
    const long long N = d.ncells;
    const long long c0 = d.off + (long long)w.a * d.nx;
    const int cnt = w.b * d.nx;
    const bool msarr = (d.flags & F_MSARR) != 0;
    const T* __restrict__ msp = msarr ? Ms + d.ms_off + (long long)w.a * d.nx : nullptr;
    const T c = (T)h6;
    for (int id = threadIdx.x; id < cnt; id += blockDim.x) {
        if (msarr && !(msp[id] > (T)0)) continue;   // no magnetisation: m stays
        const long long o = c0 + id;
        T mv[3], inc[3], out[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const long long oq = o + q * N;
            mv[q] = m[oq];
            inc[q] = c * (k1[oq] + (T)2 * k2[oq] + (T)2 * k3[oq] + k4[oq]);
        }
        if (CAY) {
            cayley_map(inc, mv, out);
        } else {
            T y[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) y[q] = mv[q] + inc[q];
            project_cell(y, out);
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) m[o + q * N] = out[q];
    }
}

static __global__ void k_c4_time(SimState* st, int nsims, double h) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nsims) st[i].t += h;
}

template <typename T, bool CAY>
static void rk4_step_impl(const Launch& L, const Rk4Buffers& B, double h) {
    cudaStream_t s = L.stream;
    const int g = L.x.count;
    const T* m = reinterpret_cast<const T*>(B.m);
    T* ys = reinterpret_cast<T*>(B.ys);
    T* H = reinterpret_cast<T*>(B.H);
    T* k[4];
    for (int j = 0; j < 4; ++j) k[j] = reinterpret_cast<T*>(B.k[j]);
    const double c[4] = {0.0, 0.5 * h, 0.5 * h, h};
    for (int st = 0; st < 4; ++st) {
        const T* y = m;
        if (st > 0) {
            k_c4_stage<T, CAY><<<g, MM_THREADS, 0, s>>>(L.desc, L.x.dev, m, k[st - 1], c[st], ys);
            y = ys;
        }
        if (CAY) {
            engine_rhs<T>(L, MODE_RHS, y, reinterpret_cast<T*>(B.dmdt), H, 0);
            k_c4_omega<T><<<g, MM_THREADS, 0, s>>>(L.desc, L.x.dev, y, H, st > 0 ? k[st - 1] : nullptr, c[st],
                                                     k[st], reinterpret_cast<const T*>(L.Ms));
        } else {
            engine_rhs<T>(L, MODE_RHS, y, k[st], nullptr, 0);   // k_s = dm/dt at the stage state
        }
    }
    k_c4_final<T, CAY><<<g, MM_THREADS, 0, s>>>(L.desc, L.x.dev, reinterpret_cast<T*>(B.m), k[0], k[1], k[2], k[3],
                                                 h / 6.0, reinterpret_cast<const T*>(L.Ms));
    k_c4_time<<<(L.nsims + 127) / 128, 128, 0, s>>>(L.state, L.nsims, h);
    if (L.launches) *L.launches += 3 + (CAY ? 4 : 0) + 2;   // stages, omega, final, time
}

template <typename T>
void rk4_step(const Launch& L, const Rk4Buffers& B, double h, bool cayley) {
    if (cayley) rk4_step_impl<T, true>(L, B, h);
    else rk4_step_impl<T, false>(L, B, h);
}

template void rk4_step<float>(const Launch&, const Rk4Buffers&, double, bool);
template void rk4_step<double>(const Launch&, const Rk4Buffers&, double, bool);

}  // namespace mm
