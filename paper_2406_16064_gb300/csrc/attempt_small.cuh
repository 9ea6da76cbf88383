// Whole Dormand-Prince attempts of small single-plane meshes in one launch.
//
// A mesh of one plane with padded FFT lengths Px, Py <= 64 (at most 32 x 32
// cells) keeps its whole integration state -- y_n, the seven stage vectors,
// the stage states and both transform stages' spectra -- in the shared
// memory of one thread-block cluster, so one cluster per simulation runs n
// attempts of the adaptive Dormand-Prince RK45 (Sec. "LLG equation") without
// leaving the chip.  CTA b of the cluster owns a block of rows and a block of
// kx columns.  Per right-hand side:
//   1. RK prologue y_s = y_n + h sum_j a_sj k_j on its rows (stage 7 also the
//      error sum sum_{j<7} e_j k_j), M = Ms y_s, zero-padded R2C along x
//      (half-length complex FFT + split, the zero upper half never read);
//   2. cluster barrier; its kx columns gathered from the peers' row spectra
//      (distributed shared memory), FFT along y (zero upper half skipped),
//      H^ = -N^ M^ per bin (Eq. 8 in Fourier space), inverse along y with
//      only the ny output rows formed;
//   3. cluster barrier; its rows gathered back from the column owners,
//      inverse C2R along x (only the nx outputs), then exchange (Eq. 5),
//      interfacial DMI (Eq. 14), uniaxial and cubic anisotropy, Zeeman and the
//      LL torque per cell, the stencil's +-y neighbours read from the peers'
//      stage states.
// The stage-1 max |dm/dt|^2 and the stage-7 error norm max |h sum e_j k_j|
// are exact maxima over ordered bits: each CTA publishes its maximum in
// shared memory and, after a barrier, every thread of every CTA reduces the
// same values in the same order, so the whole cluster takes the same
// decisions (initial step, relaxation stop, accept / reject, next h) with
// the arithmetic of k_after_stage1 and k_controller; accepted steps project
// m = y5 / |y5| per cell.  y_n and the integration state go back to global
// memory when the launch ends.
//
// Hazards between the cluster's CTAs are ordered by the two barriers of each
// right-hand side: row spectra are read by peers only between barrier A and
// B, column spectra only between B and the next A, and the stage states
// alternate between two buffers, so a CTA overwrites the buffer its
// neighbours read only after they passed the next barrier A; a last barrier
// keeps every CTA resident until no peer reads its shared memory.  There are no
// spin waits: every barrier is the hardware cluster barrier, reached the same
// number of times by every CTA since their control decisions are identical.
#pragma once
#include <cooperative_groups.h>

#include "attempt_small.h"
#include "control.cuh"

namespace mm {
namespace cg = cooperative_groups;

template <typename C>
struct SmallParams {
    using S = StoreT<C>;
    const SimDesc* __restrict__ desc;
    SimState* state;
    S* m;
    const C* __restrict__ tensor;
    const S* __restrict__ Ms;
    const V2<C>* __restrict__ tw;
    int n_attempts;
};

// RK prologue of stage ST (compile-time Dormand-Prince coefficients) on the
// CTA's n cells: ys = y_n + h sum_{j < ST-1} a_{ST,j} k_j; at ST = 7 also
// ep = sum_{j < 6} e_j k_j.  Same arithmetic, in the storage type, as k_xfwd.
template <typename S, int ST>
__device__ __forceinline__ void small_prologue(const S* yn, const S* kv, S* ys, S* ep, int cs, int n, S h) {
    const int slice = 3 * cs;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            S y = yn[c * cs + i];
            if (ST >= 2) {
                S acc = (S)0;
#pragma unroll
                for (int j = 0; j < ST - 1; ++j)
                    if (dp_a(ST, j) != 0.0) acc += (S)dp_a(ST, j) * kv[j * slice + c * cs + i];
                y += h * acc;
            }
            ys[c * cs + i] = y;
            if (ST == 7) {
                S ev = (S)0;
#pragma unroll
                for (int j = 0; j < 6; ++j)
                    if (dp_e(j) != 0.0) ev += (S)dp_e(j) * kv[j * slice + c * cs + i];
                ep[c * cs + i] = ev;
            }
        }
    }
}

// Warp-level radix-2 FFTs over groups of L = 2^l <= 32 lanes (lane j of a group
// holds element j): shuffles exchange the butterfly partners and w64 holds
// W_64^q = exp(-2 pi i q / 64), so W_{2s}^r = w64[r 32 / s].  Unnormalised.
template <typename C>
__device__ __forceinline__ C shfl_xor_v(C v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
template <>
__device__ __forceinline__ dd shfl_xor_v<dd>(dd v, int m) {
    return dd(__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m));
}
template <typename C>
__device__ __forceinline__ C shfl_idx_v(C v, int src) { return __shfl_sync(0xffffffffu, v, src); }
template <>
__device__ __forceinline__ dd shfl_idx_v<dd>(dd v, int src) {
    return dd(__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src));
}
template <typename C, bool INV>
__device__ __forceinline__ V2<C> w64_get(const V2<C>* w64, int q) {
    V2<C> w = w64[q & 63];
    if (INV) w.y = -w.y;
    return w;
}

// Decimation in frequency: natural order in, bit-reversed order out, NV
// independent sequences per lane advanced stage by stage (their shuffles and
// products overlap).
template <typename C, bool INV, int NV>
__device__ __forceinline__ void warp_dif(V2<C> (&v)[NV], int l, int j, const V2<C>* w64) {
    for (int t = l - 1; t >= 0; --t) {
        const int s = 1 << t;
        const bool up = (j & s) != 0;
        const V2<C> w = w64_get<C, INV>(w64, (j & (s - 1)) << (5 - t));
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const V2<C> u = mk<C>(shfl_xor_v(v[i].x, s), shfl_xor_v(v[i].y, s));
            v[i] = up ? cmul(u - v[i], w) : v[i] + u;
        }
    }
}

// Decimation in time: bit-reversed order in, natural order out.
template <typename C, bool INV, int NV>
__device__ __forceinline__ void warp_dit(V2<C> (&v)[NV], int l, int j, const V2<C>* w64) {
    for (int t = 0; t < l; ++t) {
        const int s = 1 << t;
        const bool up = (j & s) != 0;
        const V2<C> w = w64_get<C, INV>(w64, (j & (s - 1)) << (5 - t));
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const V2<C> u = mk<C>(shfl_xor_v(v[i].x, s), shfl_xor_v(v[i].y, s));
            const V2<C> b = cmul(up ? v[i] : u, w);
            const V2<C> a = up ? u : v[i];
            v[i] = up ? a - b : a + b;
        }
    }
}

// H^ = -N^ M^ at bin (kx, ky) of a single-plane mesh (xz = yz = 0) from the
// CTA's tensor columns ts[c][j][ky'] (c = xx, yy, zz, xy; ky' <= Py/2; xy odd in ky)
template <typename C>
__device__ __forceinline__ void small_tensor(const C* ts, int cb, int pyh, int j, int ky, int Py, V2<C>& a,
                                             V2<C>& b, V2<C>& c) {
    int kyh = ky;
    bool neg = false;
    if (ky > (Py >> 1)) { kyh = Py - ky; neg = true; }
    const C xx = ts[(0 * cb + j) * pyh + kyh], yy = ts[(1 * cb + j) * pyh + kyh];
    const C zz = ts[(2 * cb + j) * pyh + kyh];
    C xy = ts[(3 * cb + j) * pyh + kyh];
    if (neg) xy = -xy;
    const V2<C> mx = a, my = b;
    a = mk<C>(xx * mx.x + xy * my.x, xx * mx.y + xy * my.y);
    b = mk<C>(xy * mx.x + yy * my.x, xy * mx.y + yy * my.y);
    c = mk<C>(zz * c.x, zz * c.y);
}

// Column transforms per CTA: the items (kx column j, component c, half hf) --
// hf < 2 for 64-point columns, whose even and odd bins are two 32-point
// transforms, X[2k] = F32(x)[k] and X[2k+1] = F32(x W_64^n)[k] -- are spread over
// all warps, kNV per lane group.
constexpr int kNV = 3;

template <typename C>
__global__ void __launch_bounds__(kSmallThreads, 1) k_small_rk(SmallParams<C> p) {
    using S = StoreT<C>;
    using C2 = V2<C>;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ unsigned long long red_u[32];
    __shared__ unsigned long long slot[2];                // this CTA's maxima as FP64 bits
    cg::cluster_group cl = cg::this_cluster();
    const int nc = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const int sim = blockIdx.x / nc;
    const SimDesc& d = p.desc[sim];
    const int nx = d.nx, ny = d.ny, Kx = d.Kx, lPy = d.lPy, Py = d.Py, lPx = d.lPx;
    const int lX = lPx - 1, LX = 1 << lX;                 // half-length x sequences
    const int RB = small_rows_per_cta(d, nc), CB = small_cols_per_cta(d, nc);
    const int r0 = rank * RB, nr = max(0, min(ny, r0 + RB) - r0);
    const int k0 = rank * CB, nk = max(0, min(Kx, k0 + CB) - k0);
    const int cs = RB * nx, slice = 3 * cs, ncell = nr * nx;
    const int pyh = Py / 2 + 1;
    const SmallLayout lay = small_layout(d, nc, sizeof(S), sizeof(C));
    S* yn = reinterpret_cast<S*>(smraw);
    S* kv = yn + slice;
    S* ysb = kv + 7 * slice;
    S* ep = ysb + 2 * slice;
    S* hd = ep + slice;
    C2* rowX = reinterpret_cast<C2*>(smraw + lay.rows);   // [3 RB][Kx]
    C2* colH = reinterpret_cast<C2*>(smraw + lay.cols);   // [3 CB][ny]
    C2* colS = reinterpret_cast<C2*>(smraw + lay.spec);   // [3 CB][Py]
    C2* colI = reinterpret_cast<C2*>(smraw + lay.half);   // [3 CB][2][32]
    C2* w64 = reinterpret_cast<C2*>(smraw + lay.w64);
    C* ts = reinterpret_cast<C*>(smraw + lay.tens);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const long long N = d.ncells;
    S* gm = p.m + d.off + (long long)r0 * nx;
    for (int i = threadIdx.x; i < ncell; i += blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) yn[c * cs + i] = gm[c * N + i];
    }
    for (int q = threadIdx.x; q < 64; q += blockDim.x) w64[q] = p.tw[q << (MM_LOG2_LMAX - 6)];
    const bool demag = (d.flags & F_DEMAG) != 0;
    if (demag) {
        const long long plane = (long long)d.Pzh * d.Pyh * d.Kx;
        for (int i = threadIdx.x; i < 4 * nk * pyh; i += blockDim.x) {
            const int c = i / (nk * pyh), rem = i - c * nk * pyh, j = rem / pyh, ky = rem - j * pyh;
            ts[(c * CB + j) * pyh + ky] = p.tensor[d.tens_off + c * plane + (long long)ky * d.Kx + k0 + j];
        }
    }
    SimState& G = p.state[sim];
    double t = G.t, h = G.h;
    const double t_end = G.t_end, rtol = G.rtol, max_dmdt = G.max_dmdt;
    long long n_acc = G.n_acc, n_rej = G.n_rej;
    int status = G.status, accepted = 0;
    double err = G.err, maxk = G.maxk;
    unsigned long long err_bits = G.err_bits;
    cl.sync();                                  // every CTA has read the state (and its tables)

    const bool msarr = (d.flags & F_MSARR) != 0;
    const S* __restrict__ msg = msarr ? p.Ms + d.ms_off : nullptr;
    const Coef<S>& cf = coef<S>(d);
    const S mu0 = cf.mu0, inv_u = cf.inv_u, Msu = cf.Ms;
    const S ex_x = cf.ex[0], ex_y = cf.ex[1], dm_x = cf.dm[0], dm_y = cf.dm[1];
    const S cA = cf.cA, cD = cf.cD, cK = cf.cK, cC = cf.cC;
    const S ux = cf.u[0], uy = cf.u[1], uz = cf.u[2];
    const S Hx0 = cf.H[0], Hy0 = cf.H[1], Hz0 = cf.H[2];
    const S gt = cf.gt, agt = cf.agt;
    const bool prec = (d.flags & F_PREC) != 0, dmi = (d.flags & F_DMI) != 0;
    const bool do_ex = (d.flags & F_EX) != 0, do_uni = (d.flags & F_UNI) != 0, do_cub = (d.flags & F_CUB) != 0;
    const S e7 = (S)dp_e(6);
    // lane groups of the x sequences (LX lanes each)
    const int GX = 32 >> lX, gx = lane >> lX, jx = lane & (LX - 1);
    const int nseqR = 3 * nr;
    // column items: H halves of lY-point transforms, GY groups of LY lanes per warp
    const int H = lPy == 6 ? 2 : 1;
    const int lY = lPy == 6 ? 5 : lPy, LY = 1 << lY;
    const int GY = 32 >> lY, gy = lane >> lY, jy = lane & (LY - 1);
    const int nit = 3 * H * nk, nslot = (nit + GY - 1) / GY;
    const int kyb = bitrev(jy, lY);             // the bin index (within its half) lane jy holds
    bool ran = false;
    int q = 0;                                  // right-hand sides evaluated: stage-state parity

    for (int att = 0; att < p.n_attempts && status == 0; ++att) {
        ran = true;
        bool stop = false;
        for (int st = 1; st <= 7 && !stop; ++st) {
            S* ys = ysb + (q & 1) * slice;
            const S hs = (S)h;
            switch (st) {
                case 1: small_prologue<S, 1>(yn, kv, ys, ep, cs, ncell, hs); break;
                case 2: small_prologue<S, 2>(yn, kv, ys, ep, cs, ncell, hs); break;
                case 3: small_prologue<S, 3>(yn, kv, ys, ep, cs, ncell, hs); break;
                case 4: small_prologue<S, 4>(yn, kv, ys, ep, cs, ncell, hs); break;
                case 5: small_prologue<S, 5>(yn, kv, ys, ep, cs, ncell, hs); break;
                case 6: small_prologue<S, 6>(yn, kv, ys, ep, cs, ncell, hs); break;
                default: small_prologue<S, 7>(yn, kv, ys, ep, cs, ncell, hs); break;
            }
            __syncthreads();
            // ---- 1. M = Ms y_s, zero-padded R2C along x of the CTA's rows: lane n of a
            // group packs z[n] = M[2n] + i M[2n+1] (zero for 2n >= nx, so the upper half
            // is zero), FFT of length LX = Px/2, split into X_k, k = 0..LX
            if (demag) {
                for (int base = warp * GX; base < nseqR; base += nwarp * GX) {     // warp-uniform
                    const int qs = base + gx;
                    const bool valid = qs < nseqR;
                    const int r = valid ? qs / 3 : 0, c = valid ? qs - 3 * r : 0;
                    C2 z[1] = {mk<C>((C)0, (C)0)};
                    if (valid) {
#pragma unroll
                        for (int h2 = 0; h2 < 2; ++h2) {
                            const int x = 2 * jx + h2;
                            if (x < nx) {
                                const S ms = msarr ? msg[(long long)(r0 + r) * nx + x] : Msu;
                                const C mc = to_compute<C>(ms * ys[c * cs + r * nx + x]);
                                if (h2 == 0) z[0].x = mc; else z[0].y = mc;
                            }
                        }
                    }
                    warp_dif<C, false, 1>(z, lX, jx, w64);          // lane jx: Z_k, k = bitrev(jx)
                    const int k = bitrev(jx, lX);
                    const int src = (gx << lX) + bitrev((LX - k) & (LX - 1), lX);
                    const C2 Zm = cconj(mk<C>(shfl_idx_v(z[0].x, src), shfl_idx_v(z[0].y, src)));
                    const C2 E = cscale(z[0] + Zm, (C)0.5);
                    const C2 Dd = z[0] - Zm;
                    const C2 O = mk<C>(Dd.y * (C)0.5, -Dd.x * (C)0.5);
                    if (valid) {
                        C2* row = rowX + qs * Kx;
                        row[k] = E + cmul(w64_get<C, false>(w64, k << (6 - lPx)), O);
                        if (k == 0) row[LX] = E - O;
                    }
                }
            }
            cl.sync();                          // A: every row spectrum in place
            // ---- 2. columns: FFT along y of the ny non-zero rows, H^ = -N^ M^ per bin,
            // inverse along y, the ny rows kept
            if (demag) {
                for (int b0 = warp * kNV; b0 < nslot; b0 += nwarp * kNV) {           // warp-uniform
                    C2 v[kNV];
                    int it[kNV];
#pragma unroll
                    for (int u = 0; u < kNV; ++u) {
                        it[u] = (b0 + u) * GY + gy;
                        v[u] = mk<C>((C)0, (C)0);
                        if (it[u] < nit && jy < ny) {
                            const int j = it[u] / (3 * H), c = (it[u] / H) % 3, hf = it[u] % H;
                            const int ow = jy / RB;
                            v[u] = cl.map_shared_rank(rowX, ow)[(3 * (jy - ow * RB) + c) * Kx + k0 + j];
                            if (hf) v[u] = cmul(v[u], w64_get<C, false>(w64, jy));
                        }
                    }
                    warp_dif<C, false, kNV>(v, lY, jy, w64);
#pragma unroll
                    for (int u = 0; u < kNV; ++u) {
                        if (it[u] < nit) {
                            const int j = it[u] / (3 * H), c = (it[u] / H) % 3, hf = it[u] % H;
                            colS[(3 * j + c) * Py + H * kyb + hf] = v[u];
                        }
                    }
                }
                __syncthreads();
                for (int b = threadIdx.x; b < nk * Py; b += blockDim.x) {
                    const int j = b / Py, ky = b - j * Py;
                    C2* s0 = colS + 3 * j * Py + ky;
                    C2 a = s0[0], bb = s0[Py], cc = s0[2 * Py];
                    small_tensor<C>(ts, CB, pyh, j, ky, Py, a, bb, cc);
                    s0[0] = a; s0[Py] = bb; s0[2 * Py] = cc;
                }
                __syncthreads();
                for (int b0 = warp * kNV; b0 < nslot; b0 += nwarp * kNV) {
                    C2 v[kNV];
                    int it[kNV];
#pragma unroll
                    for (int u = 0; u < kNV; ++u) {
                        it[u] = (b0 + u) * GY + gy;
                        v[u] = mk<C>((C)0, (C)0);
                        if (it[u] < nit) {
                            const int j = it[u] / (3 * H), c = (it[u] / H) % 3, hf = it[u] % H;
                            v[u] = colS[(3 * j + c) * Py + H * kyb + hf];   // bit-reversed order in
                        }
                    }
                    warp_dit<C, true, kNV>(v, lY, jy, w64);                 // natural order out
#pragma unroll
                    for (int u = 0; u < kNV; ++u) {
                        if (it[u] < nit) {
                            const int j = it[u] / (3 * H), c = (it[u] / H) % 3, hf = it[u] % H;
                            if (H == 1) {
                                if (jy < ny) colH[(3 * j + c) * ny + jy] = v[u];
                            } else {
                                colI[((3 * j + c) * 2 + hf) * 32 + jy] = v[u];
                            }
                        }
                    }
                }
                if (H == 2) {
                    // x[n] = F32^-1(X[2k])[n] + W_64^-n F32^-1(X[2k+1])[n], n < ny <= 32
                    __syncthreads();
                    for (int b = threadIdx.x; b < 3 * nk * ny; b += blockDim.x) {
                        const int qc = b / ny, n = b - qc * ny;
                        colH[qc * ny + n] = colI[(2 * qc) * 32 + n] +
                                            cmul(colI[(2 * qc + 1) * 32 + n], w64_get<C, true>(w64, n));
                    }
                }
            }
            cl.sync();                          // B: every column transformed back
            // ---- 3. rows: Hermitian split and inverse C2R along x (lane j of a group
            // forms Z_k, k = bitrev(j), from the column owners' X_k and X_{LX-k}, so the
            // decimation-in-time inverse leaves z[n] in lane n: cells 2n and 2n + 1)
            if (demag) {
                for (int base = warp * GX; base < nseqR; base += nwarp * GX) {
                    const int qs = base + gx;
                    const bool valid = qs < nseqR;
                    const int r = valid ? qs / 3 : 0, c = valid ? qs - 3 * r : 0;
                    C2 z[1] = {mk<C>((C)0, (C)0)};
                    const int k = bitrev(jx, lX);
                    if (valid) {
                        const int ka = k, kb = LX - k;
                        const int oa = ka / CB, ob = kb / CB;
                        const C2 Xa = cl.map_shared_rank(colH, oa)[(3 * (ka - oa * CB) + c) * ny + r0 + r];
                        const C2 Xb = cconj(cl.map_shared_rank(colH, ob)[(3 * (kb - ob * CB) + c) * ny + r0 + r]);
                        const C2 e = Xa + Xb;
                        const C2 tq = cmul(w64_get<C, true>(w64, k << (6 - lPx)), Xa - Xb);
                        z[0] = mk<C>(e.x - tq.y, e.y + tq.x);
                    }
                    warp_dit<C, true, 1>(z, lX, jx, w64);
                    if (valid) {
                        const int x = 2 * jx;
                        if (x < nx) hd[c * cs + r * nx + x] = to_store<C>(z[0].x);
                        if (x + 1 < nx) hd[c * cs + r * nx + x + 1] = to_store<C>(z[0].y);
                    }
                }
                __syncthreads();
            }
            S* ko = kv + (st - 1) * slice;
            unsigned long long vmax = 0ull;
            for (int i = threadIdx.x; i < ncell; i += blockDim.x) {
                const int r = i / nx, x = i - r * nx, y = r0 + r;
                const S m0 = ys[i], m1 = ys[cs + i], m2 = ys[2 * cs + i];
                const S ms = msarr ? msg[(long long)y * nx + x] : Msu;
                S k0v = 0, k1v = 0, k2v = 0;
                if (ms > (S)0) {
                    const S inv = msarr ? (S)1 / (mu0 * ms) : inv_u;
                    S hd0 = 0, hd1 = 0, hd2 = 0;
                    if (demag) { hd0 = hd[i]; hd1 = hd[cs + i]; hd2 = hd[2 * cs + i]; }
                    S ex0 = 0, ex1 = 0, ex2 = 0, dm0 = 0, dm1 = 0, dm2 = 0;
                    if (do_ex || dmi) {
                        // neighbours -x, +x, -y, +y (one plane: no z neighbours); a missing
                        // one reads the cell itself and is masked
                        bool ok[4] = {x > 0, x < nx - 1, y > 0, y < ny - 1};
                        const S* rowm = ys + r * nx;
                        const S* rowl = rowm;
                        const S* rowh = rowm;
                        if (ok[2]) {
                            const int ow = (y - 1) / RB;
                            rowl = (ow == rank ? ys : cl.map_shared_rank(ys, ow)) + (y - 1 - ow * RB) * nx;
                        }
                        if (ok[3]) {
                            const int ow = (y + 1) / RB;
                            rowh = (ow == rank ? ys : cl.map_shared_rank(ys, ow)) + (y + 1 - ow * RB) * nx;
                        }
                        const int xo[4] = {ok[0] ? x - 1 : x, ok[1] ? x + 1 : x, x, x};
                        const S* rp[4] = {rowm, rowm, rowl, rowh};
                        S j0[4], j1[4], j2[4];
#pragma unroll
                        for (int nb = 0; nb < 4; ++nb) {
                            j0[nb] = rp[nb][xo[nb]];
                            j1[nb] = rp[nb][cs + xo[nb]];
                            j2[nb] = rp[nb][2 * cs + xo[nb]];
                        }
                        if (msarr) {
                            const long long cc = (long long)y * nx + x;
                            const long long moff[4] = {-1, 1, -nx, nx};
#pragma unroll
                            for (int nb = 0; nb < 4; ++nb) ok[nb] = ok[nb] && msg[cc + moff[nb]] > (S)0;
                        }
                        if (do_ex) {
                            const S fe[4] = {ex_x, ex_x, ex_y, ex_y};
#pragma unroll
                            for (int nb = 0; nb < 4; ++nb) {
                                const S f = ok[nb] ? fe[nb] : (S)0;
                                ex0 += f * (j0[nb] - m0); ex1 += f * (j1[nb] - m1); ex2 += f * (j2[nb] - m2);
                            }
                            ex0 *= cA * inv; ex1 *= cA * inv; ex2 *= cA * inv;
                        }
                        if (dmi) {
                            // sum_j e_ij x m_j / Delta: -x:-e_y, +x:+e_y, -y:+e_x, +y:-e_x
                            const S sxm = ok[0] ? -dm_x : (S)0, sxp = ok[1] ? dm_x : (S)0;
                            const S sym = ok[2] ? dm_y : (S)0, syp = ok[3] ? -dm_y : (S)0;
                            dm0 = sxm * j2[0] + sxp * j2[1];
                            dm2 = -(sxm * j0[0] + sxp * j0[1]) + sym * j1[2] + syp * j1[3];
                            dm1 = -(sym * j2[2] + syp * j2[3]);
                            dm0 *= -cD * inv; dm1 *= -cD * inv; dm2 *= -cD * inv;
                        }
                    }
                    S un0 = 0, un1 = 0, un2 = 0, cu0 = 0, cu1 = 0, cu2 = 0;
                    if (do_uni) {
                        const S mu = m0 * ux + m1 * uy + m2 * uz;
                        const S f = cK * inv * mu;
                        un0 = f * ux; un1 = f * uy; un2 = f * uz;
                    }
                    if (do_cub) {
                        const S f = -cC * inv;
                        cu0 = f * m0 * m0 * m0; cu1 = f * m1 * m1 * m1; cu2 = f * m2 * m2 * m2;
                    }
                    const S H0 = hd0 + ex0 + dm0 + un0 + cu0 + Hx0;
                    const S H1 = hd1 + ex1 + dm1 + un1 + cu1 + Hy0;
                    const S H2 = hd2 + ex2 + dm2 + un2 + cu2 + Hz0;
                    // LL form: dm/dt = -g~ m x H - alpha g~ m x (m x H)
                    const S c0 = m1 * H2 - m2 * H1, c1 = m2 * H0 - m0 * H2, c2 = m0 * H1 - m1 * H0;
                    const S dd0 = m1 * c2 - m2 * c1, dd1 = m2 * c0 - m0 * c2, dd2 = m0 * c1 - m1 * c0;
                    k0v = -agt * dd0; k1v = -agt * dd1; k2v = -agt * dd2;
                    if (prec) { k0v -= gt * c0; k1v -= gt * c1; k2v -= gt * c2; }
                }
                ko[i] = k0v; ko[cs + i] = k1v; ko[2 * cs + i] = k2v;
                if (st == 1) {
                    vmax = umax64(vmax, obits(k0v * k0v + k1v * k1v + k2v * k2v));
                } else if (st == 7) {
                    vmax = umax64(vmax, obits(fabs(fma(e7, k0v, ep[i]))));
                    vmax = umax64(vmax, obits(fabs(fma(e7, k1v, ep[cs + i]))));
                    vmax = umax64(vmax, obits(fabs(fma(e7, k2v, ep[2 * cs + i]))));
                }
            }
            ++q;
            if (st == 1 || st == 7) {
                const int si = st == 7 ? 1 : 0;
                const unsigned long long rr = block_max_u64(vmax, red_u);
                if (threadIdx.x == 0) {
                    const double v = obits_to_double<S>(rr);
                    slot[si] = (unsigned long long)__double_as_longlong(si ? fabs(h * v) : v);
                }
                cl.sync();                      // every CTA's maximum published
                unsigned long long g = 0ull;
                for (int b = 0; b < nc; ++b) g = umax64(g, *cl.map_shared_rank(&slot[si], b));
                if (st == 1) {
                    // k_after_stage1: max|dm/dt|, relaxation stop, initial step
                    const double mkv = sqrt(bits_to_double(g));
                    maxk = mkv;
                    err_bits = 0ull;
                    if (!(mkv == mkv) || isinf(mkv)) status = -4;
                    else if (max_dmdt > 0.0 && mkv < max_dmdt) status = 2;
                    else if (h <= 0.0) {
                        double h0 = mkv > 0.0 ? fmin(1e-12, 0.01 / mkv) : 1e-12;
                        if (t_end > 0.0) h0 = fmin(h0, t_end - t);
                        h = h0;
                    }
                    if (status != 0) { stop = true; accepted = 0; }
                } else {
                    // k_controller: accept when err <= 1, h <- h clamp(0.9 err^-1/5, 0.2, 5)
                    err_bits = g;
                    err = bits_to_double(g) / rtol;
                    if (!(err == err) || isinf(err)) {
                        status = -4;
                        accepted = 0;
                    } else {
                        const int acc = err <= 1.0;
                        if (acc) { t += h; n_acc += 1; } else { n_rej += 1; }
                        accepted = acc;
                        const double f = err == 0.0 ? 5.0 : fmin(5.0, fmax(0.2, 0.9 * pow(err, -0.2)));
                        h *= f;
                        if (t_end > 0.0) {
                            h = fmin(h, t_end - t);
                            if (t_end - t <= 1e-12 * t_end) status = 1;
                        }
                        if (status == 0 && !(h > 1e-24)) status = -5;
                    }
                    if (accepted) {
                        // projection m = y5 / |y5| (y5 is the stage-7 state)
                        for (int i = threadIdx.x; i < ncell; i += blockDim.x) {
                            S yv[3] = {ys[i], ys[cs + i], ys[2 * cs + i]}, mv[3];
                            project_cell(yv, mv);
                            yn[i] = mv[0]; yn[cs + i] = mv[1]; yn[2 * cs + i] = mv[2];
                        }
                        __syncthreads();
                    }
                }
            }
        }
    }
    // no CTA leaves while a peer may still read its shared memory (the maxima read after
    // the last reduction barrier)
    cl.sync();
    if (ran) {
        for (int i = threadIdx.x; i < ncell; i += blockDim.x) {
#pragma unroll
            for (int c = 0; c < 3; ++c) gm[c * N + i] = yn[c * cs + i];
        }
    }
    if (rank == 0 && threadIdx.x == 0) {
        G.t = t; G.h = h; G.n_acc = n_acc; G.n_rej = n_rej;
        G.status = status; G.accepted = accepted;
        G.err = err; G.maxk = maxk;
        G.err_bits = err_bits; G.maxk_bits = 0ull;
    }
}

template <typename C>
static cudaError_t small_prepare(size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(k_small_rk<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_small_rk<C>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

template <typename C>
static void small_config(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr, int nclusters, int nc, size_t smem,
                         cudaStream_t s) {
    cfg = {};
    cfg.gridDim = dim3((unsigned)(nclusters * nc), 1, 1);
    cfg.blockDim = dim3(kSmallThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = nc;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
}

template <typename C>
static bool small_fits_t(size_t smem, int nc) {
    if (small_prepare<C>(smem) != cudaSuccess) { cudaGetLastError(); return false; }
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    small_config<C>(cfg, attr, 1, nc, smem, nullptr);
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, k_small_rk<C>, &cfg) == cudaSuccess && ncl > 0) return true;
    cudaGetLastError();
    return false;
}

template <typename C>
static cudaError_t small_launch_t(const SmallLaunch& L) {
    using S = StoreT<C>;
    cudaError_t e = small_prepare<C>(L.smem);
    if (e != cudaSuccess) return e;
    SmallParams<C> p;
    p.desc = L.desc;
    p.state = L.state;
    p.m = reinterpret_cast<S*>(L.m);
    p.tensor = reinterpret_cast<const C*>(L.tensor);
    p.Ms = reinterpret_cast<const S*>(L.Ms);
    p.tw = reinterpret_cast<const V2<C>*>(L.tw);
    p.n_attempts = L.n_attempts;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    small_config<C>(cfg, attr, L.nsims, L.cluster, L.smem, L.stream);
    return cudaLaunchKernelEx(&cfg, k_small_rk<C>, p);
}

}  // namespace mm
