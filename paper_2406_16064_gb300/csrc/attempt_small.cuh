// Whole Dormand-Prince attempts of small single-plane meshes in one launch.
//
// A mesh of one plane with padded FFT lengths Px, Py <= 64 (at most 32 x 32
// cells) keeps its whole integration state -- y_n, the seven stage vectors,
// the stage states and both transform stages' spectra -- in the shared
// memory of one thread-block cluster, so one cluster per simulation runs n
// attempts of the adaptive Dormand-Prince RK45 (Sec. "LLG equation") without
// leaving the chip.  CTA b of the cluster owns a block of rows and a block of
// column units (a kx column, or for 64-point columns one half of it: the even
// or the odd ky bins, each a 32-point transform).  Per right-hand side:
//   1. RK prologue y_s = y_n + h sum_j a_sj k_j on its rows (stage 7 also the
//      error sum sum_{j<7} e_j k_j); the block's first and last rows stored
//      into the neighbouring CTAs' halo rows; M = Ms y_s and the zero-padded
//      R2C along x (half-length complex FFT + split), each X_k stored into the
//      shared memory of the owners of its column units (distributed shared
//      memory);
//   2. cluster barrier; per unit the FFT along y of the ny non-zero rows,
//      H^ = -N^ M^ per bin (Eq. 8 in Fourier space), the inverse along y,
//      its ny rows stored into their owners;
//   3. cluster barrier; per row the inverse C2R along x (only the nx outputs),
//      then exchange (Eq. 5), interfacial DMI (Eq. 14), uniaxial and cubic
//      anisotropy, Zeeman and the LL torque per cell, the stencil's +-y
//      neighbours from the block or its halo rows.
// Every exchange between CTAs is a store into the consumer's shared memory
// before a barrier, so every read after it is local.  The transforms are
// warp-level radix-2 FFTs: a row or column lives in the registers of a lane
// group, partners exchange by shuffles, forward transforms leave bit-reversed
// order and inverse ones take it, so no permutation is ever formed.
// The stage-1 max |dm/dt|^2 and the stage-7 error norm max |h sum e_j k_j|
// are exact maxima over ordered bits: each CTA stores its maximum into every
// CTA; after a barrier one thread per CTA reduces the same values in the same
// order and takes the decisions (initial step, relaxation stop, accept /
// reject, next h) with the arithmetic of k_after_stage1 and k_controller, so
// every CTA of the cluster takes the same ones; accepted steps project
// m = y5 / |y5| per cell.  y_n and the integration state go back to global
// memory when the launch ends.
//
// Hazards between the cluster's CTAs are ordered by the two barriers of each
// right-hand side: a CTA stores into a peer's column inputs only after the
// barrier B that follows the peer's reads of them, into its row inputs only
// after the next barrier A, and the stage states and halo rows alternate
// between two buffers by right-hand-side parity, so a buffer a neighbour reads
// is overwritten only after that neighbour passed the next barrier A; a last
// barrier keeps every CTA resident until no peer accesses its shared memory.
// There are no spin waits: every barrier is the hardware cluster barrier,
// reached the same number of times by every CTA since their control decisions
// are identical.
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
// products overlap).  Each lane forms its own output with one complex addition
// and one product: the lower lane of a pair v + u (times 1), the upper
// (u - v) w, so no lane computes both results (the product by 1 is exact in
// every compute type).
template <typename C, bool INV, int NV>
__device__ __forceinline__ void warp_dif(V2<C> (&v)[NV], int l, int j, const V2<C>* w64) {
    for (int t = l - 1; t >= 0; --t) {
        const int s = 1 << t;
        const bool up = (j & s) != 0;
        const V2<C> w = up ? w64_get<C, INV>(w64, (j & (s - 1)) << (5 - t)) : mk<C>((C)1, (C)0);
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const V2<C> u = mk<C>(shfl_xor_v(v[i].x, s), shfl_xor_v(v[i].y, s));
            const V2<C> sv = up ? mk<C>(-v[i].x, -v[i].y) : v[i];
            v[i] = cmul(u + sv, w);
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
            v[i] = a + (up ? mk<C>(-b.x, -b.y) : b);
        }
    }
}

// The step-size factor clamp(0.9 err^-1/5, 0.2, 5) of the controller, with
// err^-1/5 the root of y^-5 = err from an FP32 seed (relative error ~1e-7) by two
// Newton steps y <- y (6 - err y^5) / 5, each squaring the relative error: within
// an ulp or two of pow(err, -0.2) at a fraction of its FP64 instructions, which
// run on the FP64 pipe of one thread between two cluster barriers.  Far outside
// [(0.9/5)^5, (0.9/0.2)^5], where the clamp decides, the FP32 seed is not formed.
__device__ __forceinline__ double step_factor(double err) {
    if (err < 1e-30) return 5.0;
    if (err > 1e30) return 0.2;
    double y = (double)exp2f(-0.2f * log2f((float)err));
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const double y2 = y * y, y5 = y2 * y2 * y;
        y = y * (6.0 - err * y5) * 0.2;
    }
    return fmin(5.0, fmax(0.2, 0.9 * y));
}

// Column transforms per CTA: the items (unit j, component c) are spread over
// all warps, kNV per lane group.
constexpr int kNV = 2;

template <typename C>
__global__ void __launch_bounds__(kSmallThreads, 1) k_small_rk(SmallParams<C> p) {
    using S = StoreT<C>;
    using C2 = V2<C>;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ unsigned long long red_u[32];
    __shared__ unsigned long long slots[2][kSmallMaxCluster];   // every CTA's maxima, pushed by each CTA
    __shared__ struct {
        double t, h, err, maxk;
        unsigned long long err_bits;
        long long n_acc, n_rej;
        int status, accepted;
    } dec;                                                      // the step decision of thread 0
    cg::cluster_group cl = cg::this_cluster();
    const int nc = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const int sim = blockIdx.x / nc;
    const SimDesc& d = p.desc[sim];
    const int nx = d.nx, ny = d.ny, Kx = d.Kx, Py = d.Py, lPx = d.lPx;
    const int lX = lPx - 1, LX = 1 << lX;                 // half-length x sequences
    const int H = small_halves(d), LYh = Py / H;          // column units: halves of LYh points
    const int lY = H == 2 ? 5 : d.lPy;
    const int RB = small_rows_per_cta(d, nc), CU = small_units_per_cta(d, nc);
    const int r0 = rank * RB, nr = max(0, min(ny, r0 + RB) - r0);
    const int u0 = rank * CU, nu = max(0, min(Kx * H, u0 + CU) - u0);
    const int cs = RB * nx, slice = 3 * cs, ncell = nr * nx;
    const SmallLayout lay = small_layout(d, nc, sizeof(S), sizeof(C));
    S* yn = reinterpret_cast<S*>(smraw);
    S* kv = yn + slice;
    S* ysb = kv + 7 * slice;
    S* ep = ysb + 2 * slice;
    S* hd = ep + slice;
    S* halo = reinterpret_cast<S*>(smraw + lay.halo);     // [parity][lo, hi][3][nx]
    C2* colIn = reinterpret_cast<C2*>(smraw + lay.colin); // [3 CU][ny]
    C2* colS = reinterpret_cast<C2*>(smraw + lay.spec);   // [3 CU][LYh]
    C2* rowIn = reinterpret_cast<C2*>(smraw + lay.rowin); // [3 RB][Kx][H]
    C2* w64 = reinterpret_cast<C2*>(smraw + lay.w64);
    C* ts = reinterpret_cast<C*>(smraw + lay.tens);       // [4][CU][LYh]
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
        // tensor at the bins of the CTA's units: unit kx H + hf, bin ky = H k' + hf;
        // stored values at ky' = min(ky, Py - ky), xy odd in ky
        const long long plane = (long long)d.Pzh * d.Pyh * d.Kx;
        for (int i = threadIdx.x; i < 4 * nu * LYh; i += blockDim.x) {
            const int c = i / (nu * LYh), rem = i - c * nu * LYh, j = rem / LYh, kk = rem - j * LYh;
            const int u = u0 + j, kx = u / H, hf = u - kx * H;
            const int ky = H * kk + hf;
            const int kyh = ky > (Py >> 1) ? Py - ky : ky;
            C v = p.tensor[d.tens_off + c * plane + (long long)kyh * d.Kx + kx];
            if (c == 3 && ky > (Py >> 1)) v = -v;
            ts[(c * CU + j) * LYh + kk] = v;
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
    // lane groups of the x sequences (LX lanes each) and of the column items (LYh lanes)
    const int GX = 32 >> lX, gx = lane >> lX, jx = lane & (LX - 1);
    const int nseqR = 3 * nr;
    const int GY = 32 >> lY, gy = lane >> lY, jy = lane & (LYh - 1);
    const int nit = 3 * nu, nslot = (nit + GY - 1) / GY;
    const int LYp = small_spec_row(LYh);        // padded row of a unit's spectrum (bank spread)
    const int kyb = bitrev(jy, lY);             // the bin (within its unit) lane jy holds
    const int kyp = kyb + (kyb >> 3);           // ... at its padded position
    bool ran = false;
    int q = 0;                                  // right-hand sides evaluated: stage-state parity

    for (int att = 0; att < p.n_attempts && status == 0; ++att) {
        ran = true;
        bool stop = false;
        for (int st = 1; st <= 7 && !stop; ++st) {
            const int par = q & 1;
            S* ys = ysb + par * slice;
            S* hl = halo + par * 2 * 3 * nx;    // this parity's halo rows: [lo, hi][3][nx]
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
            // the block's first and last rows into the neighbouring CTAs' halos (the
            // row above the lower neighbour's block, the row below the upper one's)
            if ((do_ex || dmi) && nr > 0) {
                for (int i = threadIdx.x; i < 2 * 3 * nx; i += blockDim.x) {
                    const int side = i / (3 * nx), c = (i / nx) % 3, x = i % nx;
                    const int y = side == 0 ? r0 : r0 + nr - 1;           // row sent
                    const int yt = side == 0 ? y - 1 : y + 1;             // the receiver's row
                    if (yt >= 0 && yt < ny) {
                        const int ow = yt / RB;
                        // received as the receiver's hi halo (side 0) or lo halo (side 1)
                        cl.map_shared_rank(hl, ow)[((side == 0 ? 1 : 0) * 3 + c) * nx + x] =
                            ys[c * cs + (y - r0) * nx + x];
                    }
                }
            }
            // ---- 1. M = Ms y_s, zero-padded R2C along x of the CTA's rows: lane n of a
            // group packs z[n] = M[2n] + i M[2n+1] (zero for 2n >= nx, so the upper half
            // is zero), FFT of length LX = Px/2, split into X_k, k = 0..LX, each pushed to
            // the owners of its column units
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
                        const C2 Xk = E + cmul(w64_get<C, false>(w64, k << (6 - lPx)), O);
                        const C2 XL = E - O;                                // X_LX (from k = 0)
                        const int y = r0 + r;
#pragma unroll
                        for (int hf = 0; hf < 2; ++hf) {
                            if (hf < H) {
                                int u = k * H + hf, ou = u / CU;
                                cl.map_shared_rank(colIn, ou)[(3 * (u - ou * CU) + c) * ny + y] = Xk;
                                if (k == 0) {
                                    u = LX * H + hf;
                                    ou = u / CU;
                                    cl.map_shared_rank(colIn, ou)[(3 * (u - ou * CU) + c) * ny + y] = XL;
                                }
                            }
                        }
                    }
                }
            }
            cl.sync();                          // A: rows in the column owners, halos in place
            // ---- 2. column units: FFT along y of the ny non-zero rows (the odd half
            // of a 64-point column weighted by W_64^y), H^ = -N^ M^ per bin, inverse,
            // the ny rows pushed to their owners
            if (demag) {
                for (int b0 = warp * kNV; b0 < nslot; b0 += nwarp * kNV) {         // warp-uniform
                    C2 v[kNV];
                    int it[kNV];
#pragma unroll
                    for (int uu = 0; uu < kNV; ++uu) {
                        it[uu] = (b0 + uu) * GY + gy;
                        v[uu] = mk<C>((C)0, (C)0);
                        if (it[uu] < nit && jy < ny) {
                            const int j = it[uu] / 3, c = it[uu] - 3 * j;
                            v[uu] = colIn[(3 * j + c) * ny + jy];
                            if ((u0 + j) % H) v[uu] = cmul(v[uu], w64_get<C, false>(w64, jy));
                        }
                    }
                    warp_dif<C, false, kNV>(v, lY, jy, w64);
#pragma unroll
                    for (int uu = 0; uu < kNV; ++uu)
                        if (it[uu] < nit) colS[it[uu] * LYp + kyp] = v[uu];
                }
                __syncthreads();
                for (int b = threadIdx.x; b < nu * LYh; b += blockDim.x) {
                    const int j = b / LYh, kk = b - j * LYh;
                    C2* s0 = colS + 3 * j * LYp + kk + (kk >> 3);
                    const C xx = ts[(0 * CU + j) * LYh + kk], yy = ts[(1 * CU + j) * LYh + kk];
                    const C zz = ts[(2 * CU + j) * LYh + kk], xy = ts[(3 * CU + j) * LYh + kk];
                    const C2 mx = s0[0], my = s0[LYp], mz = s0[2 * LYp];
                    s0[0] = mk<C>(xx * mx.x + xy * my.x, xx * mx.y + xy * my.y);
                    s0[LYp] = mk<C>(xy * mx.x + yy * my.x, xy * mx.y + yy * my.y);
                    s0[2 * LYp] = mk<C>(zz * mz.x, zz * mz.y);
                }
                __syncthreads();
                for (int b0 = warp * kNV; b0 < nslot; b0 += nwarp * kNV) {
                    C2 v[kNV];
                    int it[kNV];
#pragma unroll
                    for (int uu = 0; uu < kNV; ++uu) {
                        it[uu] = (b0 + uu) * GY + gy;
                        v[uu] = it[uu] < nit ? colS[it[uu] * LYp + kyp] : mk<C>((C)0, (C)0);   // bit-reversed in
                    }
                    warp_dit<C, true, kNV>(v, lY, jy, w64);                 // natural order out
#pragma unroll
                    for (int uu = 0; uu < kNV; ++uu) {
                        if (it[uu] < nit && jy < ny) {
                            const int j = it[uu] / 3, c = it[uu] - 3 * j;
                            const int u = u0 + j, kx = u / H, hf = u - kx * H;
                            const int ow = jy / RB;
                            cl.map_shared_rank(rowIn, ow)[((3 * (jy - ow * RB) + c) * Kx + kx) * H + hf] = v[uu];
                        }
                    }
                }
            }
            cl.sync();                          // B: every column result in its row owner
            // ---- 3. rows: X(kx) = the units' results (the odd half weighted by W_64^-y),
            // Hermitian split and inverse C2R along x (lane j of a group forms Z_k,
            // k = bitrev(j), so the decimation-in-time inverse leaves z[n] in lane n:
            // cells 2n and 2n + 1)
            if (demag) {
                for (int base = warp * GX; base < nseqR; base += nwarp * GX) {
                    const int qs = base + gx;
                    const bool valid = qs < nseqR;
                    const int r = valid ? qs / 3 : 0;
                    C2 z[1] = {mk<C>((C)0, (C)0)};
                    const int k = bitrev(jx, lX);
                    if (valid) {
                        const C2* ri = rowIn + qs * Kx * H;
                        C2 Xa, Xb;
                        if (H == 2) {
                            const C2 wy = w64_get<C, true>(w64, r0 + r);
                            Xa = ri[2 * k] + cmul(ri[2 * k + 1], wy);
                            Xb = ri[2 * (LX - k)] + cmul(ri[2 * (LX - k) + 1], wy);
                        } else {
                            Xa = ri[k];
                            Xb = ri[LX - k];
                        }
                        Xb = cconj(Xb);
                        const C2 e = Xa + Xb;
                        const C2 tq = cmul(w64_get<C, true>(w64, k << (6 - lPx)), Xa - Xb);
                        z[0] = mk<C>(e.x - tq.y, e.y + tq.x);
                    }
                    warp_dit<C, true, 1>(z, lX, jx, w64);
                    if (valid) {
                        const int c = qs - 3 * r, x = 2 * jx;
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
                        // neighbours -x, +x, -y, +y (one plane: no z neighbours) from the
                        // CTA's rows or its halo rows; a missing one reads the cell itself and
                        // is masked.  Component stride: cs in the block, nx in a halo.
                        bool ok[4] = {x > 0, x < nx - 1, y > 0, y < ny - 1};
                        const S* rowm = ys + r * nx;
                        const S* rowl = rowm;
                        const S* rowh = rowm;
                        int csl = cs, csh = cs;
                        if (ok[2]) {
                            if (r > 0) rowl = rowm - nx;
                            else { rowl = hl; csl = nx; }
                        }
                        if (ok[3]) {
                            if (r < nr - 1) rowh = rowm + nx;
                            else { rowh = hl + 3 * nx; csh = nx; }
                        }
                        const int xo[4] = {ok[0] ? x - 1 : x, ok[1] ? x + 1 : x, x, x};
                        const S* rp[4] = {rowm, rowm, rowl, rowh};
                        const int cst[4] = {cs, cs, csl, csh};
                        S j0[4], j1[4], j2[4];
#pragma unroll
                        for (int nb = 0; nb < 4; ++nb) {
                            j0[nb] = rp[nb][xo[nb]];
                            j1[nb] = rp[nb][cst[nb] + xo[nb]];
                            j2[nb] = rp[nb][2 * cst[nb] + xo[nb]];
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
                    // the field in the order hd + ex + dm + un + cu + H_ext, terms that are
                    // switched off left out (adding their zeros changes no bit; FP64
                    // additions are what the FP64 epilogue spends its pipe on)
                    S H0 = hd0, H1 = hd1, H2 = hd2;
                    if (do_ex) { H0 += ex0; H1 += ex1; H2 += ex2; }
                    if (dmi) { H0 += dm0; H1 += dm1; H2 += dm2; }
                    if (do_uni) { H0 += un0; H1 += un1; H2 += un2; }
                    if (do_cub) { H0 += cu0; H1 += cu1; H2 += cu2; }
                    H0 += Hx0; H1 += Hy0; H2 += Hz0;
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
                    const unsigned long long vb = (unsigned long long)__double_as_longlong(si ? fabs(h * v) : v);
                    for (int b = 0; b < nc; ++b) cl.map_shared_rank(&slots[si][0], b)[rank] = vb;
                }
                cl.sync();                      // every CTA's maximum in every CTA
                // one thread takes the step decision (its FP64 arithmetic, pow included, would
                // otherwise run in every warp on the FP64 pipe) and broadcasts it
                if (threadIdx.x == 0) {
                    unsigned long long g = 0ull;
                    for (int b = 0; b < nc; ++b) g = umax64(g, slots[si][b]);
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
                        if (status != 0) accepted = 0;
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
                            const double f = step_factor(err);
                            h *= f;
                            if (t_end > 0.0) {
                                h = fmin(h, t_end - t);
                                if (t_end - t <= 1e-12 * t_end) status = 1;
                            }
                            if (status == 0 && !(h > 1e-24)) status = -5;
                        }
                    }
                    dec.t = t; dec.h = h; dec.err = err; dec.maxk = maxk; dec.err_bits = err_bits;
                    dec.n_acc = n_acc; dec.n_rej = n_rej; dec.status = status; dec.accepted = accepted;
                }
                __syncthreads();
                t = dec.t; h = dec.h; err = dec.err; maxk = dec.maxk; err_bits = dec.err_bits;
                n_acc = dec.n_acc; n_rej = dec.n_rej; status = dec.status; accepted = dec.accepted;
                if (st == 1) {
                    if (status != 0) stop = true;
                } else {
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
    // no CTA leaves before every peer is past its last access to the cluster's shared
    // memory
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
