// Extended local terms of the x-inverse epilogue (k_xinv<T, E, true>), for
// simulations with F_EXT:
//   DMI of every symmetry class (Sec. "Dzyaloshinskii-Moriya Energy"):
//     H_i = -1/(mu0 Ms_i) sum_j D_ij (e_ij x m_j) / Delta_ij with e_ij for the
//     neighbours (-x, +x, -y, +y, -z, +z): interfacial (-e_y, e_y, e_x, -e_x),
//     bulk r_ij = (-e_x, e_x, -e_y, e_y, -e_z, e_z), D_2d (e_x, -e_x, -e_y, e_y);
//   exchange and DMI with per-cell constants, A_ij = 2 A_i A_j / (A_i + A_j)
//     and D_ij alike (0 where the two values sum to 0) (Sec. "Exchange energy");
//   spin torques (Sec. "Spin transfer torques"): T = m x (m x G) + beta m x G
//     - a_J m x (m x p) - b_J m x p with G = (u.grad)m by central differences
//     (a neighbour outside the mesh or without magnetisation is the cell
//     itself), added to the LL right-hand side as (T + alpha m x T)/(1 + alpha^2),
//     the solution of the implicit equation's extra part.
// Free boundaries and Ms = 0 neighbours are dropped from the sums exactly as
// in the standard epilogue.
#pragma once
#include "mm_kernels.cuh"

namespace mm {

// DMI vector of neighbour nb (-x, +x, -y, +y, -z, +z) of class kind as
// +-(axis + 1) (axis 0, 1, 2 = x, y, z), 0 where the class has none
__device__ __forceinline__ int dmi_code(int kind, int nb) {
    switch (kind) {
        case 1: return nb == 0 ? -2 : nb == 1 ? 2 : nb == 2 ? 1 : nb == 3 ? -1 : 0;
        case 2: return nb == 0 ? -1 : nb == 1 ? 1 : nb == 2 ? -2 : nb == 3 ? 2 : nb == 4 ? -3 : 3;
        case 3: return nb == 0 ? 1 : nb == 1 ? -1 : nb == 2 ? -2 : nb == 3 ? 2 : 0;
        default: return 0;
    }
}

template <typename T>
__device__ __forceinline__ T harmonic_pair(T a, T b) {
    const T s = a + b;
    return s != (T)0 ? (T)2 * a * b / s : (T)0;
}

// Exchange (ex, scaled by 1/(mu0 Ms) through inv), DMI (dm) and (u.grad)m (g)
// of one cell.  acp / dcp: the tile's per-cell A and D (nullptr: uniform).
template <typename T>
__device__ __forceinline__ void ext_local(const SimDesc& d, const Coef<T>& cf, const ExtCoef<T>& xc,
                                          const T* __restrict__ m0p, const T* __restrict__ m1p,
                                          const T* __restrict__ m2p, const T* __restrict__ msp,
                                          const T* __restrict__ acp, const T* __restrict__ dcp, int cell, int x,
                                          int y, int z, T m0, T m1, T m2, T inv, T (&ex)[3], T (&dm)[3],
                                          T (&g)[3]) {
    const int nx = d.nx, ny = d.ny, nz = d.nz, sz = nx * ny;
    bool ok[6] = {x > 0, x < nx - 1, y > 0, y < ny - 1, z > 0, z < nz - 1};
    const int off[6] = {-1, 1, -nx, nx, -sz, sz};
    T j0[6], j1[6], j2[6];
#pragma unroll
    for (int nb = 0; nb < 6; ++nb) {
        const int o = cell + (ok[nb] ? off[nb] : 0);
        j0[nb] = m0p[o]; j1[nb] = m1p[o]; j2[nb] = m2p[o];
    }
    if (msp) {
#pragma unroll
        for (int nb = 0; nb < 6; ++nb) ok[nb] = ok[nb] && msp[cell + (ok[nb] ? off[nb] : 0)] > (T)0;
    }
    if (d.flags & F_EX) {
        const T fe[6] = {cf.ex[0], cf.ex[0], cf.ex[1], cf.ex[1], cf.ex[2], cf.ex[2]};
        const T Ai = acp ? acp[cell] : xc.A;
#pragma unroll
        for (int nb = 0; nb < 6; ++nb) {
            const T Aij = acp ? harmonic_pair(Ai, acp[cell + (ok[nb] ? off[nb] : 0)]) : Ai;
            const T f = ok[nb] ? fe[nb] * Aij : (T)0;
            ex[0] += f * (j0[nb] - m0); ex[1] += f * (j1[nb] - m1); ex[2] += f * (j2[nb] - m2);
        }
        const T c = (T)2 * inv;
        ex[0] *= c; ex[1] *= c; ex[2] *= c;
    }
    if (d.flags & F_DMI) {
        const T dinv[3] = {cf.dm[0], cf.dm[1], xc.dinv_z};
        const T Di = dcp ? dcp[cell] : xc.D;
#pragma unroll
        for (int nb = 0; nb < 6; ++nb) {
            const int code = dmi_code(d.dmi_kind, nb);       // uniform over the simulation
            if (code == 0) continue;
            const T Dij = dcp ? harmonic_pair(Di, dcp[cell + (ok[nb] ? off[nb] : 0)]) : Di;
            const T f = ok[nb] ? (code > 0 ? Dij : -Dij) * dinv[nb >> 1] : (T)0;
            const int a = (code > 0 ? code : -code) - 1;
            // e_x x m = (0, -mz, my), e_y x m = (mz, 0, -mx), e_z x m = (-my, mx, 0)
            if (a == 0) { dm[1] -= f * j2[nb]; dm[2] += f * j1[nb]; }
            else if (a == 1) { dm[0] += f * j2[nb]; dm[2] -= f * j0[nb]; }
            else { dm[0] -= f * j1[nb]; dm[1] += f * j0[nb]; }
        }
        dm[0] *= -inv; dm[1] *= -inv; dm[2] *= -inv;
    }
    if (d.eflags & E_STT) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int lo = 2 * a, hi = 2 * a + 1;
            const T u = xc.gu[a];
            g[0] += u * ((ok[hi] ? j0[hi] : m0) - (ok[lo] ? j0[lo] : m0));
            g[1] += u * ((ok[hi] ? j1[hi] : m1) - (ok[lo] ? j1[lo] : m1));
            g[2] += u * ((ok[hi] ? j2[hi] : m2) - (ok[lo] ? j2[lo] : m2));
        }
    }
}

// k += (T + alpha m x T) / (1 + alpha^2) for the spin torques T of the cell
template <typename T>
__device__ __forceinline__ void ext_torque(const SimDesc& d, const ExtCoef<T>& xc, T m0, T m1, T m2,
                                           const T (&g)[3], T& k0, T& k1, T& k2) {
    T t0 = 0, t1 = 0, t2 = 0;
    if (d.eflags & E_STT) {
        const T a0 = m1 * g[2] - m2 * g[1], a1 = m2 * g[0] - m0 * g[2], a2 = m0 * g[1] - m1 * g[0];
        const T b0 = m1 * a2 - m2 * a1, b1 = m2 * a0 - m0 * a2, b2 = m0 * a1 - m1 * a0;
        t0 += b0 + xc.beta * a0; t1 += b1 + xc.beta * a1; t2 += b2 + xc.beta * a2;
    }
    if (d.eflags & E_SOT) {
        const T p0 = xc.p[0], p1 = xc.p[1], p2 = xc.p[2];
        const T a0 = m1 * p2 - m2 * p1, a1 = m2 * p0 - m0 * p2, a2 = m0 * p1 - m1 * p0;
        const T b0 = m1 * a2 - m2 * a1, b1 = m2 * a0 - m0 * a2, b2 = m0 * a1 - m1 * a0;
        t0 -= xc.aJ * b0 + xc.bJ * a0; t1 -= xc.aJ * b1 + xc.bJ * a1; t2 -= xc.aJ * b2 + xc.bJ * a2;
    }
    const T c0 = m1 * t2 - m2 * t1, c1 = m2 * t0 - m0 * t2, c2 = m0 * t1 - m1 * t0;
    k0 += (t0 + xc.alpha * c0) * xc.inv_q;
    k1 += (t1 + xc.alpha * c1) * xc.inv_q;
    k2 += (t2 + xc.alpha * c2) * xc.inv_q;
}

}  // namespace mm
