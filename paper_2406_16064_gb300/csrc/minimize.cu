// Steepest-descent energy minimisation with Barzilai-Borwein steps
// (Sec. "Steepest descent energy minimization").  Per cell, with
// f = m x H_eff(m) and g = m x (m x H_eff(m)), the paper's norm-preserving step
//     (1 + tau^2 |f|^2 / 4) m_{k+1} = (1 - tau^2 |f|^2 / 4) m_k - tau g_k
// and the step-size rules tau^1 = sum s.s / sum s.y, tau^2 = sum s.y / sum y.y
// (s = m_k - m_{k-1}, y = g_k - g_{k-1}, sums over one simulation's cells).
// Readings where the paper is silent: the rules alternate (tau^1 on odd steps,
// tau^2 on even ones), tau_0 = 0.01 / max |g|, a rule that is not positive and
// finite (negative curvature along the last step) falls back to 0.01 / max |g|,
// every step is capped at tau <= 1 / max |g| (no cell turns by more than about
// one radian; without the cap random starts never settle), and a simulation
// stops once the max |dm/dt| of its LL right-hand side at m_k drops below the
// threshold.
//
// One step of a batch = the effective-field passes of the right-hand side
// (H_eff written) and three kernels:
//   k_sd_reduce  g = m x (m x H); s, y; per simulation s.s, s.y, y.y
//                (compensated per thread, FP64 across threads) and the exact
//                max |g|^2 (ordered bits); g_prev <- g
//   k_sd_tau     per simulation, FP64: stopping test, tau_k
//   k_sd_update  m_{k+1} from the explicit form (|f| = |g| for |m| = 1), then
//                the norm-restoring projection (the update keeps |m| only in
//                exact arithmetic); m_prev <- m_k; cells with Ms = 0 stay
#include "control.cuh"
#include "minimize.h"

namespace mm {

template <typename T>
__device__ __forceinline__ void cross3(const T (&a)[3], const T (&b)[3], T (&c)[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

template <typename T>
__global__ void __launch_bounds__(MM_THREADS) k_sd_reduce(const SimDesc* __restrict__ desc, SdState* sd,
                                                          const WorkItem* __restrict__ items, const T* m,
                                                          const T* H, const T* mprev, T* gprev,
                                                          const T* __restrict__ Ms) {
    __shared__ double red[MM_THREADS / 32];
    __shared__ unsigned long long redu[MM_THREADS / 32];
    const WorkItem w = items[blockIdx.x];
    SdState& S = sd[w.sim];
    if (S.status != 0) return;                     // uniform over the CTA
    const SimDesc& d = desc[w.sim];
    const long long N = d.ncells;
    const long long c0 = d.off + (long long)w.a * d.nx;
    const int cnt = w.b * d.nx;
    const bool msarr = (d.flags & F_MSARR) != 0;
    const T* __restrict__ msp = msarr ? Ms + d.ms_off + (long long)w.a * d.nx : nullptr;
    CSum<T> ss, sy, yy;
    unsigned long long gmax = 0ull;
    for (int id = threadIdx.x; id < cnt; id += blockDim.x) {
        const long long o = c0 + id;
        T mv[3], Hv[3], g[3] = {(T)0, (T)0, (T)0};
#pragma unroll
        for (int c = 0; c < 3; ++c) { mv[c] = m[o + c * N]; Hv[c] = H[o + c * N]; }
        if (!msarr || msp[id] > (T)0) {
            T f[3];
            cross3(mv, Hv, f);
            cross3(mv, f, g);
        }
        T s2 = 0, sdy = 0, y2 = 0, g2 = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const T s = mv[c] - mprev[o + c * N];
            const T y = g[c] - gprev[o + c * N];
            s2 += s * s;
            sdy += s * y;
            y2 += y * y;
            g2 += g[c] * g[c];
            gprev[o + c * N] = g[c];
        }
        ss.add(s2);
        sy.add(sdy);
        yy.add(y2);
        gmax = umax64(gmax, obits(g2));
    }
    const double a = block_csum(ss, red);
    if (threadIdx.x == 0) atomicAdd(&S.ss, a);
    const double b = block_csum(sy, red);
    if (threadIdx.x == 0) atomicAdd(&S.sy, b);
    const double c = block_csum(yy, red);
    if (threadIdx.x == 0) atomicAdd(&S.yy, c);
    const unsigned long long r = block_max_u64(gmax, redu);
    if (threadIdx.x == 0)
        atomicMax(&S.maxg_bits, (unsigned long long)__double_as_longlong(obits_to_double<T>(r)));
}

static __global__ void k_sd_tau(SdState* sd, int nsims) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nsims) return;
    SdState& S = sd[i];
    if (S.status != 0) return;
    const double maxg = sqrt(bits_to_double(S.maxg_bits));
    S.max_dmdt = maxg * S.dmdt_scale;
    if (!(maxg == maxg) || isinf(maxg)) { S.status = -4; return; }
    if (S.stop_dmdt > 0.0 && S.max_dmdt < S.stop_dmdt) { S.status = 2; return; }
    const double safe = maxg > 0.0 ? 0.01 / maxg : 0.0;
    if (S.k == 0) {
        S.tau = safe;
    } else {
        const double cand = (S.k & 1) ? S.ss / S.sy : S.sy / S.yy;
        S.tau = (cand > 0.0 && !isinf(cand)) ? cand : safe;   // NaN takes the safe step too
    }
    if (maxg > 0.0) S.tau = fmin(S.tau, 1.0 / maxg);         // at most ~1 rad a step
    S.k += 1;
    S.ss = 0.0;
    S.sy = 0.0;
    S.yy = 0.0;
    S.maxg_bits = 0ull;
}

template <typename T>
__global__ void __launch_bounds__(MM_THREADS) k_sd_update(const SimDesc* __restrict__ desc, const SdState* sd,
                                                          const WorkItem* __restrict__ items, T* m, T* mprev,
                                                          const T* g, const T* __restrict__ Ms) {
    const WorkItem w = items[blockIdx.x];
    const SdState& S = sd[w.sim];
    if (S.status != 0) return;
    const SimDesc& d = desc[w.sim];
    const long long N = d.ncells;
    const long long c0 = d.off + (long long)w.a * d.nx;
    const int cnt = w.b * d.nx;
    const bool msarr = (d.flags & F_MSARR) != 0;
    const T* __restrict__ msp = msarr ? Ms + d.ms_off + (long long)w.a * d.nx : nullptr;
    const T tau = (T)S.tau;
    for (int id = threadIdx.x; id < cnt; id += blockDim.x) {
        const long long o = c0 + id;
        T mv[3], gv[3], mn[3], mr[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) { mv[c] = m[o + c * N]; gv[c] = g[o + c * N]; }
#pragma unroll
        for (int c = 0; c < 3; ++c) mprev[o + c * N] = mv[c];
        if (msarr && !(msp[id] > (T)0)) continue;   // no magnetisation: m stays
        const T a = (T)0.25 * tau * tau * (gv[0] * gv[0] + gv[1] * gv[1] + gv[2] * gv[2]);
        const T inv = (T)1 / ((T)1 + a);
#pragma unroll
        for (int c = 0; c < 3; ++c) mn[c] = (((T)1 - a) * mv[c] - tau * gv[c]) * inv;
        project_cell(mn, mr);
#pragma unroll
        for (int c = 0; c < 3; ++c) m[o + c * N] = mr[c];
    }
}

template <typename T>
void sd_step(const Launch& L, const SdBuffers& B) {
    cudaStream_t s = L.stream;
    engine_rhs<T>(L, MODE_RHS, reinterpret_cast<const T*>(B.m), reinterpret_cast<T*>(B.dmdt),
                  reinterpret_cast<T*>(B.H), 0);
    const T* Ms = reinterpret_cast<const T*>(L.Ms);
    k_sd_reduce<T><<<L.x.count, MM_THREADS, 0, s>>>(L.desc, B.sd, L.x.dev, reinterpret_cast<const T*>(B.m),
                                                     reinterpret_cast<const T*>(B.H),
                                                     reinterpret_cast<const T*>(B.mprev),
                                                     reinterpret_cast<T*>(B.gprev), Ms);
    k_sd_tau<<<(L.nsims + 127) / 128, 128, 0, s>>>(B.sd, L.nsims);
    k_sd_update<T><<<L.x.count, MM_THREADS, 0, s>>>(L.desc, B.sd, L.x.dev, reinterpret_cast<T*>(B.m),
                                                     reinterpret_cast<T*>(B.mprev),
                                                     reinterpret_cast<const T*>(B.gprev), Ms);
    if (L.launches) *L.launches += 3;
}

template void sd_step<float>(const Launch&, const SdBuffers&);
template void sd_step<double>(const Launch&, const SdBuffers&);

}  // namespace mm
