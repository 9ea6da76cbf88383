// Pass kernels of one LLG right-hand-side evaluation over a batch of
// simulations (one launch per pass covers every simulation of the batch,
// one CTA -- or one thread-block cluster -- per work item):
//
//   k_xfwd   RK stage prologue y_s = y_n + h sum_j a_sj k_j (Dormand-Prince,
//            Sec. "LLG equation"), M = Ms y_s, zero-padded real-to-complex
//            FFT along x (half-length complex FFT + split), for the ny*nz
//            non-zero rows only.
//   k_ycol   column FFTs along y over blocks of kx columns: forward (only the
//            ny non-zero input rows are read), inverse (only ny output rows
//            written), or -- for films (Pz = 1) -- forward, tensor product,
//            inverse in one kernel.
//   k_zcol   forward FFT along z, tensor product H^ = -N^ M^ (Eq. 8 in
//            Fourier space), inverse FFT along z; nz of Pz planes in/out
//            (meshes with nz > 8).
//   k_yzc    thin films (1 < nz <= 8): one thread-block cluster of nz CTAs per
//            kx block, CTA z owning plane z.  Each CTA transforms its plane
//            along y; after a cluster barrier every CTA takes a share of the
//            ky rows, gathers the nz planes from its peers' shared memory
//            (distributed shared memory), convolves them along z directly
//            with the tensor of the x-y transformed Newell kernel (Eq. 8 with
//            the z sum written out), and scatters the nz planes back; after a
//            second barrier each CTA inverts its plane along y.  Replaces
//            y forward + z + y inverse.
//   k_xinv   complex-to-real inverse FFT along x (only the nx outputs), then
//            per cell: exchange (Eq. 5), interfacial DMI (Eq. 14), uniaxial
//            and cubic anisotropy, Zeeman, the LL torque (LL form of the
//            LLG equation), optional H_eff, the stage-1 max|dm/dt| and the
//            stage-7 embedded error norm (ordered-bit max reductions, scaled
//            and combined in FP64), or the energies (compensated per-thread
//            sums, FP64 across threads) in energy mode; the extended variant
//            adds bulk / D_2d DMI, per-cell A and D and the spin torques
//            (ext_terms.cuh).
#pragma once
#include <cooperative_groups.h>

#include "ext_terms.cuh"
#include "mm_kernels.cuh"

namespace mm {

static constexpr double kMu0 = 4e-7 * 3.14159265358979323846;

// spectrum element (c, z, y, kx) in the kx-blocked layout [3][nz][NBx][Py][Ty]
template <typename T>
__device__ __forceinline__ long long spec_index(const SimDesc& d, int c, int z, int y, int kx) {
    return d.spec_off + (((((long long)c * d.nz + z) * d.NBx + (kx >> d.lTy)) * d.Py + y) << d.lTy) +
           (kx & (d.Ty - 1));
}

// first element of block b of plane (c, z); element (y, j) sits at + y*Ty + j
template <typename T>
__device__ __forceinline__ long long spec_block(const SimDesc& d, int c, int z, int b) {
    return d.spec_off + ((((long long)c * d.nz + z) * d.NBx + b) * d.Py << d.lTy);
}

// H = T M with T the stored (negated, scaled) tensor at bin (kx, ky, kz)
template <typename T>
__device__ __forceinline__ void tensor_apply(const SimDesc& d, const T* __restrict__ tens, int kx, int ky,
                                             int kz, V2<T>& Mx, V2<T>& My, V2<T>& Mz) {
    int kyh = ky, kzh = kz;
    T sy = (T)1, sz = (T)1;
    if (ky > (d.Py >> 1)) { kyh = d.Py - ky; sy = (T)-1; }
    if (kz > (d.Pz >> 1)) { kzh = d.Pz - kz; sz = (T)-1; }
    const long long plane = (long long)d.Pzh * d.Pyh * d.Kx;
    const long long i0 = d.tens_off + ((long long)kzh * d.Pyh + kyh) * d.Kx + kx;
    const T xx = tens[i0], yy = tens[i0 + plane], zz = tens[i0 + 2 * plane];
    const T xy = sy * tens[i0 + 3 * plane];
    T xz = (T)0, yz = (T)0;
    if (d.ncomp == 6) { xz = sz * tens[i0 + 4 * plane]; yz = sy * sz * tens[i0 + 5 * plane]; }
    const V2<T> a = Mx, b = My, c = Mz;
    Mx = mk<T>(xx * a.x + xy * b.x + xz * c.x, xx * a.y + xy * b.y + xz * c.y);
    My = mk<T>(xy * a.x + yy * b.x + yz * c.x, xy * a.y + yy * b.y + yz * c.y);
    Mz = mk<T>(xz * a.x + yz * b.x + zz * c.x, xz * a.y + yz * b.y + zz * c.y);
}

template <typename T>
__device__ __forceinline__ bool sim_inactive(const PassParams<T>& p, int sim) {
    return (p.mode == MODE_RK || p.mode == MODE_NEB) && p.state[sim].status != 0;
}

// ---------------------------------------------------------------- x forward
// Shared memory: two buffers of 3*nrows padded sequences (pidx) of Lh complex
// values, sequence q = 3 r + c (row r of the tile, component c).
// S: Dormand-Prince stage of the RK prologue (2..7), or 0 for none (stage 1
// and the non-RK modes).  The stage's coefficients are compile-time
// constants, so zero ones vanish and the stage vectors' loads issue together.
template <typename T, int S>
__global__ void __launch_bounds__(MM_XTHREADS_MAX<T>, 1) k_xfwd(PassParams<T> p) {
    using R = StoreT<T>;                         // the RK prologue runs in the storage type
    extern __shared__ __align__(16) unsigned char smraw[];
    const WorkItem w = p.items[blockIdx.x];
    if (sim_inactive(p, w.sim)) return;
    const SimDesc& d = p.desc[w.sim];
    const int nx = d.nx, ny = d.ny;
    const long long N = d.ncells;
    const int lLh = d.lPx - 1, Lh = 1 << lLh;
    const int SL = padded_len(Lh);
    const int row0 = w.a, nrows = w.b;
    const int nseq = 3 * nrows;
    V2<T>* bufA = reinterpret_cast<V2<T>*>(smraw);
    V2<T>* bufB = bufA + nseq * SL;
    const long long base = d.off - p.off_adjust + (long long)row0 * nx;   // first cell of the tile
    const bool demag = (d.flags & F_DEMAG) != 0;
    const bool msarr = (d.flags & F_MSARR) != 0;
    const R hstep = (R)((p.mode == MODE_RK || p.mode == MODE_NEB) ? p.state[w.sim].h : 0.0);
    const R* __restrict__ msp = msarr ? p.Ms + d.ms_off + (long long)row0 * nx : nullptr;
    // z[n] = M[2n] + i M[2n+1] is non-zero for n < ceil(nx/2) <= Lh/2 (Lh >= nx): only the
    // lower half of each sequence is stored, the first FFT stage does not read the upper half
    const int lhalf = lLh > 0 ? lLh - 1 : 0;
    const int tot = nrows << lhalf;
    const R* __restrict__ mp = p.m + base;
    R* __restrict__ yp = p.ybuf + base;
    R* __restrict__ ep = p.errp + base;
    for (int id = threadIdx.x; id < tot; id += blockDim.x) {
        const int r = id >> lhalf, n = id & ((1 << lhalf) - 1);
        V2<T> val[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) val[c] = mk<T>((T)0, (T)0);
        // both cells' state and stage vectors are loaded before any is combined or stored,
        // so all loads of the item are in flight together; a stage vector the stage's
        // coefficients or (stage 7) error weights use is loaded once for both
        R yv[2][3];
        R kv[6][2][3];
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
            const int x = 2 * n + h2;
            if (x < nx) {
                const int cell = r * nx + x;                   // within the tile
#pragma unroll
                for (int c = 0; c < 3; ++c) yv[h2][c] = mp[c * N + cell];
#pragma unroll
                for (int j = 0; j < 6; ++j) {
                    if (j < S - 1 && (dp_a(S, j) != 0.0 || (S == 7 && dp_e(j) != 0.0))) {
                        const R* __restrict__ kj = p.kvec[j] + base + cell;
#pragma unroll
                        for (int c = 0; c < 3; ++c) kv[j][h2][c] = kj[c * N];
                    }
                }
            }
        }
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
            const int x = 2 * n + h2;
            if (x < nx) {
                const int cell = r * nx + x;                   // within the tile
                R yvv[3] = {yv[h2][0], yv[h2][1], yv[h2][2]};
                if (S >= 2) {
                    R acc[3] = {(R)0, (R)0, (R)0};
#pragma unroll
                    for (int j = 0; j < S - 1; ++j) {
                        if (dp_a(S, j) != 0.0) {
                            const R aj = (R)dp_a(S, j);
#pragma unroll
                            for (int c = 0; c < 3; ++c) acc[c] += aj * kv[j][h2][c];
                        }
                    }
#pragma unroll
                    for (int c = 0; c < 3; ++c) yvv[c] += hstep * acc[c];
#pragma unroll
                    for (int c = 0; c < 3; ++c) yp[c * N + cell] = yvv[c];
                    if (S == 7) {
                        R ev[3] = {(R)0, (R)0, (R)0};
#pragma unroll
                        for (int j = 0; j < 6; ++j) {
                            if (dp_e(j) != 0.0) {
                                const R ej = (R)dp_e(j);
#pragma unroll
                                for (int c = 0; c < 3; ++c) ev[c] += ej * kv[j][h2][c];
                            }
                        }
#pragma unroll
                        for (int c = 0; c < 3; ++c) ep[c * N + cell] = ev[c];
                    }
                }
                if (demag) {
                    const R ms = msarr ? msp[cell] : coef<R>(d).Ms;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const T mc = to_compute<T>(ms * yvv[c]);
                        if (h2 == 0) val[c].x = mc; else val[c].y = mc;
                    }
                }
            }
        }
        if (demag) {
            const int pos = ix<true>(n, 1);
#pragma unroll
            for (int c = 0; c < 3; ++c) bufA[(3 * r + c) * SL + pos] = val[c];
        }
    }
    if (!demag) return;
    __syncthreads();
    const V2<T>* Z = stockham_fft<T, false, (sizeof(T) == 4 ? 4 : 3), true, false>(bufA, bufB, lLh, nseq, SL, p.tw);
    const V2<T>* __restrict__ wsplit = p.tw + MM_LMAX + stw_base(1, d.lPx);   // W_Px^k, k < Lh
    // split the half-length transform into X_k, k = 0..Lh, and store in the kx-blocked layout
    const int z0 = row0 / ny, y0 = row0 - z0 * ny;       // a tile never crosses a plane
    V2<T>* sp = p.spec + d.spec_off;
    const int lT = d.lTy, TT = d.Ty;
    const int plane = d.NBx * (d.Py << lT);               // elements of one (c, z) plane
    // X_k and X_{Lh-k} come from the same two half-length bins: with E_k, O_k the even
    // and odd parts at k, E_{Lh-k} = conj(E_k) and O_{Lh-k} = conj(O_k), so one work
    // item loads Z_k and Z_{Lh-k} once and writes both outputs (k = 0..Lh/2)
    const int lhl = lLh > 0 ? lLh - 1 : 0;
    const int hl = lLh > 0 ? 1 << lhl : 0;
    const int totp = lLh > 0 ? nseq << lhl : 0;
    for (int id = threadIdx.x; id < totp + nseq; id += blockDim.x) {
        int q, k;
        if (id < totp) { q = id >> lhl; k = id & (hl - 1); } else { q = id - totp; k = hl; }
        const int kp = Lh - k;
        const int r = q / 3, c = q - 3 * r;
        const int y = y0 + r, z = z0;
        const V2<T>* s = Z + q * SL;
        const V2<T> Zk = s[ix<true>(k & (Lh - 1), 1)];
        const V2<T> Zm = cconj(s[ix<true>(kp & (Lh - 1), 1)]);
        const V2<T> E = cscale(Zk + Zm, (T)0.5);
        const V2<T> Dd = Zk - Zm;
        const V2<T> O = mk<T>(Dd.y * (T)0.5, -Dd.x * (T)0.5);
        V2<T>* so = sp + (c * d.nz + z) * plane + (y << lT);
        so[((k >> lT) * d.Py << lT) + (k & (TT - 1))] = E + cmul(k < Lh ? wsplit[k] : mk<T>((T)-1, (T)0), O);
        if (kp != k)
            so[((kp >> lT) * d.Py << lT) + (kp & (TT - 1))] =
                cconj(E) + cmul(kp < Lh ? wsplit[kp] : mk<T>((T)-1, (T)0), cconj(O));
    }
}

// ---------------------------------------------------------------- y columns
// YMODE 0: forward (one component), 1: inverse (one component),
//       2: forward + tensor product + inverse (three components, Pz == 1)
// A CTA owns one kx block (Ty columns) of one plane.  Shared memory holds the
// block as rows [y][cc][col] (row stride NC*Ty).  The forward is a
// decimation-in-frequency FFT (natural order in, bit-reversed out) and the
// inverse a decimation-in-time FFT (bit-reversed in, natural out), so neither
// needs a permutation: the spectrum between them is in bit-reversed row
// order, in shared memory (YMODE 2) or in the global spectrum (YMODE 0 -> z
// pass -> YMODE 1), and the tensor product reads bin ky = bitrev(row).
template <typename T, int YMODE>
__global__ void __launch_bounds__(MM_XTHREADS_MAX<T>, 1) k_ycol(PassParams<T> p) {
    extern __shared__ __align__(16) unsigned char smraw[];
    V2<T>* sm = reinterpret_cast<V2<T>*>(smraw);
    const WorkItem w = p.items[blockIdx.x];
    if (sim_inactive(p, w.sim)) return;
    const SimDesc& d = p.desc[w.sim];
    const int L = d.Py, lL = d.lPy, TT = d.Ty, lT = d.lTy, ny = d.ny;
    const int z = w.a, b = w.b;
    const int kx0 = b << lT;
    const int ncols = min(TT, d.Kx - kx0);
    constexpr int NC = (YMODE == 2) ? 3 : 1;
    const int c0 = (YMODE == 2) ? 0 : w.c;
    const int es = NC * TT;
    long long gb[NC];
#pragma unroll
    for (int cc = 0; cc < NC; ++cc) gb[cc] = spec_block<T>(d, c0 + cc, z, b);
    const int nload = (YMODE == 1) ? L : ny;
    constexpr int VPC = 16 / (int)sizeof(V2<T>);                 // complex values per 16-byte copy
    if ((TT % VPC) == 0) {
        // rows y < nload as 16-byte async copies; rows nload <= y < L/2 zeroed (the
        // forward's first group does not read the upper half; the inverse loads all rows)
        const int cpr = TT / VPC, ncp = NC * nload * cpr;
        for (int i = threadIdx.x; i < ncp; i += blockDim.x) {
            const int q = i % cpr, yc = i / cpr;
            const int cc = yc % NC, y = yc / NC;
            cp_async16(sm + y * es + cc * TT + q * VPC, p.spec + gb[cc] + ((long long)y << lT) + q * VPC);
        }
        const int zrows = (YMODE == 1) ? 0 : (L >> 1) - nload;
        for (int i = threadIdx.x; i < zrows * es; i += blockDim.x) sm[nload * es + i] = mk<T>((T)0, (T)0);
        cp_async_wait_all();
    } else {
        for (int b0 = threadIdx.x; b0 < (L << lT); b0 += 4 * blockDim.x) {   // 4 NC loads in flight
            V2<T> v[NC][4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int id = b0 + u * blockDim.x;
                const int y = id >> lT;
#pragma unroll
                for (int cc = 0; cc < NC; ++cc)
                    v[cc][u] = (id < (L << lT) && y < nload) ? p.spec[gb[cc] + id] : mk<T>((T)0, (T)0);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int id = b0 + u * blockDim.x;
                if (id < (L << lT)) {
                    const int col = id & (TT - 1), y = id >> lT;
#pragma unroll
                    for (int cc = 0; cc < NC; ++cc) sm[y * es + cc * TT + col] = v[cc][u];
                }
            }
        }
    }
    __syncthreads();
    if (YMODE == 0) {
        fft_dif<T, false, false, true>(sm, lL, es, 1, es, p.tw);
        for (int id = threadIdx.x; id < (L << lT); id += blockDim.x)
            p.spec[gb[0] + id] = sm[id];             // NC == 1: row stride Ty
        return;
    }
    if (YMODE == 2) {
        fft_dif<T, false, false, true>(sm, lL, es, 1, es, p.tw);
        for (int id = threadIdx.x; id < (L << lT); id += blockDim.x) {
            const int col = id & (TT - 1), r = id >> lT;
            if (col < ncols) {
                V2<T>* q = sm + r * es + col;
                V2<T> a = q[0], bb = q[TT], c = q[2 * TT];
                tensor_apply<T>(d, p.tensor, kx0 + col, bitrev(r, lL), 0, a, bb, c);
                q[0] = a; q[TT] = bb; q[2 * TT] = c;
            }
        }
        __syncthreads();
    }
    fft_dit<T, true, false, true>(sm, lL, es, 1, es, p.tw);
#pragma unroll
    for (int cc = 0; cc < NC; ++cc) {
        for (int id = threadIdx.x; id < (ny << lT); id += blockDim.x) {
            const int col = id & (TT - 1), y = id >> lT;
            p.spec[gb[cc] + id] = sm[y * es + cc * TT + col];
        }
    }
}

// ---------------------------------------------------------------- z columns
// One CTA per (global row, kx block): the three components' z columns, rows
// [z][c][col] (row stride 3*Ty).  Forward decimation in frequency, the
// tensor product at kz = bitrev(row), inverse decimation in time.  The y pass
// before it leaves the rows of each plane in bit-reversed order, so global
// row w.a holds bin ky = bitrev(w.a) (Py = 1: row 0, bin 0).
template <typename T>
__global__ void __launch_bounds__(MM_XTHREADS_MAX<T>, 1) k_zcol(PassParams<T> p) {
    extern __shared__ __align__(16) unsigned char smraw[];
    V2<T>* sm = reinterpret_cast<V2<T>*>(smraw);
    const WorkItem w = p.items[blockIdx.x];
    if (sim_inactive(p, w.sim)) return;
    const SimDesc& d = p.desc[w.sim];
    const int L = d.Pz, lL = d.lPz, TT = d.Ty, lT = d.lTy, nz = d.nz;
    const int row = w.a, b = w.b;
    const int ky = bitrev(row, d.lPy);
    const int kx0 = b << lT;
    const int ncols = min(TT, d.Kx - kx0);
    const int es = 3 * TT;
    constexpr int VPC = 16 / (int)sizeof(V2<T>);                 // complex values per 16-byte copy
    if ((TT % VPC) == 0) {
        // planes z < nz: one Ty-wide run per (z, c) as 16-byte async copies; planes
        // nz <= z < L/2 zeroed (the forward's first group does not read the upper half)
        const int cpr = TT / VPC, ncp = nz * 3 * cpr;
        for (int i = threadIdx.x; i < ncp; i += blockDim.x) {
            const int q = i % cpr, zc = i / cpr;
            const int c = zc % 3, z = zc / 3;
            cp_async16(sm + z * es + c * TT + q * VPC,
                       p.spec + spec_block<T>(d, c, z, b) + ((long long)row << lT) + q * VPC);
        }
        for (int i = threadIdx.x; i < ((L >> 1) - nz) * es; i += blockDim.x) sm[nz * es + i] = mk<T>((T)0, (T)0);
        cp_async_wait_all();
    } else {
        const int tot = (L * 3) << lT;
        for (int b0 = threadIdx.x; b0 < tot; b0 += 4 * blockDim.x) {   // four loads in flight
            V2<T> v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int id = b0 + u * blockDim.x;
                const int col = id & (TT - 1);
                const int rest = id >> lT;
                const int c = rest % 3;
                const int z = rest / 3;
                v[u] = (id < tot && z < nz) ? p.spec[spec_block<T>(d, c, z, b) + ((long long)row << lT) + col]
                                            : mk<T>((T)0, (T)0);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int id = b0 + u * blockDim.x;
                if (id < tot) {
                    const int col = id & (TT - 1);
                    const int rest = id >> lT;
                    const int c = rest % 3;
                    const int z = rest / 3;
                    sm[z * es + c * TT + col] = v[u];
                }
            }
        }
    }
    __syncthreads();
    fft_dif<T, false, false, true>(sm, lL, es, 1, es, p.tw);
    for (int id = threadIdx.x; id < (L << lT); id += blockDim.x) {
        const int col = id & (TT - 1);
        const int r = id >> lT;
        if (col < ncols) {
            V2<T>* q = sm + r * es + col;
            V2<T> a = q[0], bb = q[TT], c = q[2 * TT];
            tensor_apply<T>(d, p.tensor, kx0 + col, ky, bitrev(r, lL), a, bb, c);
            q[0] = a; q[TT] = bb; q[2 * TT] = c;
        }
    }
    __syncthreads();
    fft_dit<T, true, false, true>(sm, lL, es, 1, es, p.tw);
    const int tot3 = (nz * 3) << lT;
    for (int id = threadIdx.x; id < tot3; id += blockDim.x) {
        const int col = id & (TT - 1);
        const int rest = id >> lT;
        const int c = rest % 3;
        const int z = rest / 3;
        p.spec[spec_block<T>(d, c, z, b) + ((long long)row << lT) + col] = sm[z * es + c * TT + col];
    }
}

// ------------------------------------------------ y + z fused, cluster per block
// QP tensor values of one (column, ky) bin of the blocked layout, as 16-byte loads
// (q must be 16-byte aligned: a bin's first value, or an offset of 16 bytes from it)
template <int QP>
__device__ __forceinline__ void load_bin(const float* __restrict__ q, float (&v)[QP]) {
    static_assert(QP % 4 == 0, "FP32 bins are loaded as whole float4s");
    const float4* q4 = reinterpret_cast<const float4*>(q);
#pragma unroll
    for (int i = 0; i < QP / 4; ++i) {
        const float4 t = __ldg(q4 + i);
        v[4 * i] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
    }
}
template <int QP>
__device__ __forceinline__ void load_bin(const double* __restrict__ q, double (&v)[QP]) {
    static_assert(QP % 2 == 0, "FP64 bins are loaded as whole double2s");
    const double2* q2 = reinterpret_cast<const double2*>(q);
#pragma unroll
    for (int i = 0; i < QP / 2; ++i) {
        const double2 t = __ldg(q2 + i);
        v[2 * i] = t.x; v[2 * i + 1] = t.y;
    }
}

template <int QP>
__device__ __forceinline__ void load_bin(const dd* __restrict__ q, dd (&v)[QP]) {
    static_assert(QP % 2 == 0, "double-float bins are loaded as whole float4s");
    const float4* q4 = reinterpret_cast<const float4*>(q);
#pragma unroll
    for (int i = 0; i < QP / 2; ++i) {
        const float4 t = __ldg(q4 + i);
        v[2 * i] = dd(t.x, t.y); v[2 * i + 1] = dd(t.z, t.w);
    }
}

// z step of the cluster pass: for every (ky row, kx column) of this CTA's
// share, gather the NZ planes' values from the cluster's shared memories and
// convolve along z directly, H(z) = sum_z' N^(kx, ky, z - z') M(z') (Eq. 8 with
// the z sum written out: for NZ <= 8 planes this costs fewer operations than a
// zero-padded length-2 NZ FFT pair plus the product), then scatter H back.
// The stored tensor holds dz >= 0; negative offsets follow from the z parities
// (xz, yz odd); xz and yz are imaginary in (kx, ky, dz) and stored as t with
// N^ = i t; the ky fold flips xy and yz.
// LOWREG: the per-plane form below also for 4-byte types (the builds bounded for 3 or
// 4 CTAs per SM).
template <typename T, int NZ, bool LOWREG = false>
__device__ void yzc_zstep(const PassParams<T>& p, const SimDesc& d, V2<T>* const (&rem)[8], int rank, int es,
                          int b, int ncols) {
    constexpr int QP = yzc_qp(NZ);
    const int TT = d.Ty, lT = d.lTy, Py = d.Py;
    const int ky_lo = (int)(((long long)rank * Py) / NZ);    // share of rows
    const int ky_hi = (int)(((long long)(rank + 1) * Py) / NZ);
    const int nwork = (ky_hi - ky_lo) << lT;
    const T* __restrict__ tb = p.tensor + d.tens_off + (long long)b * d.Pyh * TT * QP;
    for (int id = threadIdx.x; id < nwork; id += blockDim.x) {
        const int col = id & (TT - 1);
        const int r = ky_lo + (id >> lT);              // row of the bit-reversed y spectrum
        const int ky = bitrev(r, d.lPy);
        if (col >= ncols) continue;
        const bool fy = ky > (Py >> 1);
        const int kyh = fy ? Py - ky : ky;
        const T sy = fy ? (T)-1 : (T)1;
        const int o = r * es + col;
        const T* __restrict__ tq = tb + ((long long)kyh * TT + col) * QP;
        V2<T> M[NZ][3];
#pragma unroll
        for (int z = 0; z < NZ; ++z) {
#pragma unroll
            for (int c = 0; c < 3; ++c) M[z][c] = rem[z][o + c * TT];
        }
        if constexpr (NZ >= 6) {
            // many planes: offsets dz outermost, so only one offset's six tensor
            // values are live next to the NZ accumulators
            V2<T> H[NZ][3];
#pragma unroll
            for (int z = 0; z < NZ; ++z) {
#pragma unroll
                for (int c = 0; c < 3; ++c) H[z][c] = mk<T>((T)0, (T)0);
            }
#pragma unroll
            for (int dz = 0; dz < NZ; ++dz) {
                const T* t = tq + 6 * dz;
                const T xx = t[0], yy = t[1], zz = t[2], xy = sy * t[3], xzp = t[4], yzp = sy * t[5];
#pragma unroll
                for (int sgn = 0; sgn < 2; ++sgn) {
                    if (sgn == 1 && dz == 0) continue;
                    const T xz = sgn ? -xzp : xzp, yz = sgn ? -yzp : yzp;   // odd in z
#pragma unroll
                    for (int z2 = 0; z2 + dz < NZ; ++z2) {
                        // sgn 0: z = z2 + dz (offset +dz); sgn 1: z = z2, source z2 + dz (offset -dz)
                        const int z = sgn ? z2 : z2 + dz, zs = sgn ? z2 + dz : z2;
                        const V2<T> a = M[zs][0], bb = M[zs][1], c = M[zs][2];
                        H[z][0].x += xx * a.x + xy * bb.x - xz * c.y;
                        H[z][0].y += xx * a.y + xy * bb.y + xz * c.x;
                        H[z][1].x += xy * a.x + yy * bb.x - yz * c.y;
                        H[z][1].y += xy * a.y + yy * bb.y + yz * c.x;
                        H[z][2].x += zz * c.x - xz * a.y - yz * bb.y;
                        H[z][2].y += zz * c.y + xz * a.x + yz * bb.x;
                    }
                }
            }
#pragma unroll
            for (int z = 0; z < NZ; ++z) {
#pragma unroll
                for (int c = 0; c < 3; ++c) rem[z][o + c * TT] = H[z][c];
            }
            continue;
        }
        if constexpr (sizeof(T) == 8 || LOWREG) {
            // 8-byte types (FP64, double-float): one output plane at a time, each offset's
            // six tensor values loaded where they are used (L1), so the NZ planes of M and
            // one plane of accumulators are what stays in registers (the plane loop is not
            // unrolled, so no other plane's tensor loads are hoisted next to it)
#pragma unroll 1
            for (int z = 0; z < NZ; ++z) {
                V2<T> H0 = mk<T>((T)0, (T)0), H1 = H0, H2 = H0;
#pragma unroll
                for (int z2 = 0; z2 < NZ; ++z2) {
                    const int dz = z - z2 >= 0 ? z - z2 : z2 - z;
                    const T so = z - z2 >= 0 ? (T)1 : (T)-1;    // xz, yz odd in z
                    T t[6];
                    if constexpr (sizeof(T) == 8) {
                        load_bin<6>(tq + 6 * dz, t);            // 48-byte offsets: 16-byte aligned
                    } else {
#pragma unroll
                        for (int i = 0; i < 6; ++i) t[i] = __ldg(tq + 6 * dz + i);   // 24-byte offsets
                    }
                    const T xx = t[0], yy = t[1], zz = t[2], xy = sy * t[3];
                    const T xz = so * t[4], yz = so * sy * t[5];
                    const V2<T> a = M[z2][0], bb = M[z2][1], c = M[z2][2];
                    H0.x += xx * a.x + xy * bb.x - xz * c.y;
                    H0.y += xx * a.y + xy * bb.y + xz * c.x;
                    H1.x += xy * a.x + yy * bb.x - yz * c.y;
                    H1.y += xy * a.y + yy * bb.y + yz * c.x;
                    H2.x += zz * c.x - xz * a.y - yz * bb.y;
                    H2.y += zz * c.y + xz * a.x + yz * bb.x;
                }
                rem[z][o] = H0;
                rem[z][o + TT] = H1;
                rem[z][o + 2 * TT] = H2;
            }
            continue;
        }
        T tv[QP];
        load_bin<QP>(tq, tv);
#pragma unroll
        for (int z = 0; z < NZ; ++z) {
            V2<T> H0 = mk<T>((T)0, (T)0), H1 = H0, H2 = H0;
#pragma unroll
            for (int z2 = 0; z2 < NZ; ++z2) {
                const int dz = z - z2 >= 0 ? z - z2 : z2 - z;
                const T so = z - z2 >= 0 ? (T)1 : (T)-1;        // xz, yz odd in z
                const T* t = tv + 6 * dz;
                const T xx = t[0], yy = t[1], zz = t[2], xy = sy * t[3];
                const T xz = so * t[4], yz = so * sy * t[5];     // N^xz = i xz, N^yz = i yz
                const V2<T> a = M[z2][0], bb = M[z2][1], c = M[z2][2];
                H0.x += xx * a.x + xy * bb.x - xz * c.y;
                H0.y += xx * a.y + xy * bb.y + xz * c.x;
                H1.x += xy * a.x + yy * bb.x - yz * c.y;
                H1.y += xy * a.y + yy * bb.y + yz * c.x;
                H2.x += zz * c.x - xz * a.y - yz * bb.y;
                H2.y += zz * c.y + xz * a.x + yz * bb.x;
            }
            rem[z][o] = H0;
            rem[z][o + TT] = H1;
            rem[z][o + 2 * TT] = H2;
        }
    }
}

// Two CTAs per SM (128 registers a thread): FP32, and FP64 up to 4 planes (a
// small spill there costs less than the halved occupancy, measured on the
// 512x512x4 film); FP64 with more planes keeps the registers it needs.
// NZ: planes (= cluster size); WIDE: 32-point register groups for the y columns
// (FP32; see plan_yzc_list); MINB: CTAs per SM the build is bounded for (0: the
// rule above; 3: 85 registers a thread, 4: 64 registers and 8-point column
// groups, for narrow column tiles whose shared memory lets that many CTAs share
// an SM).
template <typename T, int NZ, bool WIDE, int MINB = 0>
__global__ void __launch_bounds__(MM_THREADS, MINB ? MINB : ((sizeof(T) == 4 || NZ <= 4) ? 2 : 1))
    k_yzc(PassParams<T> p) {
    namespace cg = cooperative_groups;
    extern __shared__ __align__(16) unsigned char smraw[];
    V2<T>* sm = reinterpret_cast<V2<T>*>(smraw);
    cg::cluster_group cl = cg::this_cluster();
    const int ncl = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const WorkItem w = p.items[blockIdx.x / ncl];
    if (sim_inactive(p, w.sim)) return;          // uniform over the cluster: one simulation per cluster
    const SimDesc& d = p.desc[w.sim];
    const int L = d.Py, lL = d.lPy, TT = d.Ty, lT = d.lTy, ny = d.ny, nz = d.nz;
    const int z = rank, b = w.b;
    const int kx0 = b << lT;
    const int ncols = min(TT, d.Kx - kx0);
    const int es = 3 * TT;                      // rows [y][c][col] at y * es
    long long gb[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) gb[c] = spec_block<T>(d, c, z, b);
    // rows y < ny from the spectrum, ny <= y < L/2 zero; the upper half (L >= 2 ny) is not
    // stored: the forward's first register group does not read it
    const int nld = (L >> 1) << lT;
    for (int b0 = threadIdx.x; b0 < nld; b0 += 4 * blockDim.x) {   // 12 loads in flight
        V2<T> v[3][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int id = b0 + u * blockDim.x;
            const int y = id >> lT;
#pragma unroll
            for (int c = 0; c < 3; ++c)
                v[c][u] = (id < nld && y < ny) ? p.spec[gb[c] + id] : mk<T>((T)0, (T)0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int id = b0 + u * blockDim.x;
            if (id < nld) {
                const int col = id & (TT - 1), y = id >> lT;
#pragma unroll
                for (int c = 0; c < 3; ++c) sm[y * es + c * TT + col] = v[c][u];
            }
        }
    }
    __syncthreads();
    constexpr int GMC = MINB >= 4 ? 3 : (WIDE && sizeof(T) == 4) ? 5 : kGroupMax<T>;
    fft_dif<T, false, false, true, GMC>(sm, lL, es, 1, es, p.tw);   // rows leave in bit-reversed order
    cl.sync();                                  // every plane transformed along y
    V2<T>* rem[8];
#pragma unroll
    for (int zz = 0; zz < 8; ++zz) rem[zz] = zz < nz ? cl.map_shared_rank(sm, zz) : sm;
    yzc_zstep<T, NZ, (MINB >= 3)>(p, d, rem, rank, es, b, ncols);   // NZ == d.nz, fixed per launch
    cl.sync();                                  // every row back in its owner's plane
    fft_dit<T, true, false, true, GMC>(sm, lL, es, 1, es, p.tw);    // bit-reversed in, natural out
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        for (int id = threadIdx.x; id < (ny << lT); id += blockDim.x) {
            const int col = id & (TT - 1), y = id >> lT;
            p.spec[gb[c] + id] = sm[y * es + c * TT + col];
        }
    }
}

// ------------------------------------------------------- x inverse + fields
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
    return a > b ? a : b;
}

__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long v, unsigned long long* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = umax64(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    unsigned long long r = 0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r = umax64(r, red[i]);
    }
    return r;
}

// Shared memory: two buffers of 3*nrows padded sequences of Kx complex values.
// ENERGY: energy accumulation (energy and NEB modes) instead of the RK reductions.
// EXT: the extended variant, launched when some simulation of the batch has
// F_EXT (ext_terms.cuh); its other simulations take the standard path.
template <typename T, bool ENERGY, bool EXT>
__global__ void __launch_bounds__(MM_XTHREADS_MAX<T>, 1) k_xinv(PassParams<T> p, const StoreT<T>* __restrict__ ys) {
    using R = StoreT<T>;                         // the epilogue runs in the storage type
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ unsigned long long red_u[32];
    __shared__ double red_e[ENERGY ? 6 * 32 : 1];
    const WorkItem w = p.items[blockIdx.x];
    if (sim_inactive(p, w.sim)) return;
    const SimDesc& d = p.desc[w.sim];
    const int nx = d.nx, ny = d.ny, nz = d.nz;
    const long long N = d.ncells;
    const int lLh = d.lPx - 1, Lh = 1 << lLh, Kx = d.Kx;
    const int SK = padded_len(Kx);
    const int row0 = w.a, nrows = w.b;
    const int nseq = 3 * nrows;
    V2<T>* bufA = reinterpret_cast<V2<T>*>(smraw);
    V2<T>* bufB = bufA + nseq * SK;
    const bool demag = (d.flags & F_DEMAG) != 0;
    const bool msarr = (d.flags & F_MSARR) != 0;
    const int z0 = row0 / ny, y0 = row0 - z0 * ny;      // a tile never crosses a plane
    const long long tile = d.off - p.off_adjust + (long long)row0 * nx;
    const bool ext = EXT && (d.flags & F_EXT) != 0;
    // Staged state rows (F_XSTAGE): the tile's rows y0-1 .. y0+nrows of its plane and its
    // rows of the planes below and above, as bulk copies issued now and completed on an
    // mbarrier while the inverse FFT runs; the epilogue then reads m and its six
    // neighbours from shared memory.  Taken only where every run starts on a 16-byte
    // boundary and is a multiple of 16 bytes (rows of nx * sizeof(R) bytes), uniformly
    // for the CTA; otherwise the epilogue loads them from global memory.
    __shared__ __align__(8) unsigned long long xbar;
    const int ylo = y0 > 0 ? y0 - 1 : 0, yhi = y0 + nrows < ny ? y0 + nrows : ny - 1;
    const int prow = yhi - ylo + 1;
    const bool zlo = z0 > 0, zhi = z0 + 1 < nz;
    const size_t rowb = (size_t)nx * sizeof(R);
    const R* __restrict__ gstate = ys + (d.off - p.off_adjust);
    R* stg = reinterpret_cast<R*>(smraw + xinv_stage_offset(nseq, SK, sizeof(V2<T>)));
    const bool staged = (d.flags & F_XSTAGE) != 0 && !ext && rowb % 16 == 0 &&
                        reinterpret_cast<uintptr_t>(gstate) % 16 == 0;
    if (staged) {
        if (threadIdx.x == 0) mbar_init(&xbar, 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            // per component: its prow plane rows, then nrows rows below, nrows rows above
            const unsigned pb = (unsigned)(prow * rowb), zb = (unsigned)(nrows * rowb);
            mbar_expect_tx(&xbar, 3 * pb + (zlo ? 3 * zb : 0) + (zhi ? 3 * zb : 0));
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const R* gc = gstate + c * N;
                R* sc = stg + c * (prow + 2 * nrows) * nx;
                bulk_g2s(sc, gc + ((long long)z0 * ny + ylo) * nx, pb, &xbar);
                if (zlo) bulk_g2s(sc + prow * nx, gc + ((long long)(z0 - 1) * ny + y0) * nx, zb, &xbar);
                if (zhi) bulk_g2s(sc + (prow + nrows) * nx, gc + ((long long)(z0 + 1) * ny + y0) * nx, zb, &xbar);
            }
        }
    }
    const V2<T>* Hd = nullptr;
    if (demag) {
        const V2<T>* sp = p.spec + d.spec_off;
        const int lT = d.lTy, TT = d.Ty;
        const int plane = d.NBx * (d.Py << lT);
        const int tot1 = nseq << lLh;
        // four loads in flight per thread before their shared-memory stores
        for (int b0 = threadIdx.x; b0 < tot1 + nseq; b0 += 4 * blockDim.x) {
            V2<T> v[4];
            int dst[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int id = b0 + u * blockDim.x;
                dst[u] = -1;
                if (id < tot1 + nseq) {
                    int q, k;
                    if (id < tot1) { q = id >> lLh; k = id & (Lh - 1); } else { q = id - tot1; k = Lh; }
                    const int r = q / 3, c = q - 3 * r;
                    const int o = (c * nz + z0) * plane + (((k >> lT) * d.Py + y0 + r) << lT) + (k & (TT - 1));
                    v[u] = sp[o];
                    dst[u] = q * SK + ix<true>(k, 1);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (dst[u] >= 0) bufA[dst[u]] = v[u];
        }
        __syncthreads();
        if (d.Py == 1 && d.Pz == 1) {            // x is the only transformed axis
            for (int id = threadIdx.x; id < nrows * Kx; id += blockDim.x) {
                const int r = id / Kx, k = id - r * Kx;
                const int pk = ix<true>(k, 1);
                V2<T>* s0 = bufA + (3 * r + 0) * SK;
                V2<T>* s1 = bufA + (3 * r + 1) * SK;
                V2<T>* s2 = bufA + (3 * r + 2) * SK;
                V2<T> a = s0[pk], b = s1[pk], c = s2[pk];
                tensor_apply<T>(d, p.tensor, k, 0, 0, a, b, c);
                s0[pk] = a; s1[pk] = b; s2[pk] = c;
            }
            __syncthreads();
        }
        // Hermitian split into B: Z_k = (X_k + X*_{Lh-k}) + i W^{-k} (X_k - X*_{Lh-k}), k < Lh
        const V2<T>* __restrict__ wsplit = p.tw + MM_LMAX + stw_base(1, d.lPx);   // W_Px^k, k < Lh
        for (int id = threadIdx.x; id < tot1; id += blockDim.x) {
            const int q = id >> lLh, k = id & (Lh - 1);
            const V2<T>* s = bufA + q * SK;
            const V2<T> Xa = s[ix<true>(k, 1)], Xb = cconj(s[ix<true>(Lh - k, 1)]);
            const V2<T> e = Xa + Xb;
            const V2<T> t = cmul(stw_get<T, true>(wsplit, k), Xa - Xb);
            bufB[q * SK + ix<true>(k, 1)] = mk<T>(e.x - t.y, e.y + t.x);
        }
        __syncthreads();
        // only z[n], n < ceil(nx/2) <= Lh/2, is read by the epilogue: the last stage
        // writes the lower half of each sequence
        Hd = stockham_fft<T, true, (sizeof(T) == 4 ? 4 : 3), false, true>(bufB, bufA, lLh, nseq, SK, p.tw);
    }

    // per-cell local fields and torque; coefficients precomputed in the context
    // precision (no FP64 arithmetic per thread in an FP32 context)
    const Coef<R>& cf = coef<R>(d);
    const R mu0 = cf.mu0, inv_u = cf.inv_u;
    const R ex_x = cf.ex[0], ex_y = cf.ex[1], ex_z = cf.ex[2];
    const R dm_x = cf.dm[0], dm_y = cf.dm[1];
    const R cA = cf.cA, cD = cf.cD, cK = cf.cK, cC = cf.cC;
    const R ux = cf.u[0], uy = cf.u[1], uz = cf.u[2];
    const R Hx0 = cf.H[0], Hy0 = cf.H[1], Hz0 = cf.H[2];
    const R gt = cf.gt, agt = cf.agt, Msu = cf.Ms;
    const bool prec = (d.flags & F_PREC) != 0;
    const bool dmi = (d.flags & F_DMI) != 0;
    const bool do_ex = (d.flags & F_EX) != 0, do_uni = (d.flags & F_UNI) != 0, do_cub = (d.flags & F_CUB) != 0;
    const bool write_k = !ENERGY;
    const int sz = nx * ny;
    // m of the tile's cells (index r nx + x) and of their +-z neighbours: the staged rows,
    // or the state in global memory
    const R* __restrict__ m0p = ys + tile;
    long long cs = N;                            // component stride
    int dzb = -sz, dza = sz;                     // offsets of the -z and +z neighbours
    if (staged) {
        // a copy that has not landed after a bounded wait is reported (MM_ETIMEOUT),
        // waited for once more (it writes this CTA's shared memory) and the tile skipped
        const bool late = !mbar_wait_bounded(&xbar, 0, 1 << 20);
        if (__syncthreads_or(late)) {
            if (threadIdx.x == 0) atomicExch(&p.state[w.sim].status, -6);
            mbar_wait_bounded(&xbar, 0, 1 << 20);
            return;
        }
        m0p = stg + (y0 - ylo) * nx;
        cs = (long long)(prow + 2 * nrows) * nx;
        dzb = (prow - (y0 - ylo)) * nx;
        dza = dzb + nrows * nx;
    }
    const R* __restrict__ m1p = m0p + cs;
    const R* __restrict__ m2p = m1p + cs;
    const R* __restrict__ msp = msarr ? p.Ms + d.ms_off + (long long)row0 * nx : nullptr;
    const R* __restrict__ acp = (ext && (d.eflags & E_CELL)) ? p.cellp + d.cell_off + (long long)row0 * nx : nullptr;
    const R* __restrict__ dcp = acp ? acp + N : nullptr;
    const R e7 = (R)dp_e(6);
    const bool red1 = !ENERGY && p.mode == MODE_RK && p.stage == 1;
    const bool red7 = !ENERGY && p.mode == MODE_RK && p.stage == 7;
    unsigned long long vmax = 0ull;
    CSum<R> esum[6];
    for (int r = 0; r < nrows; ++r) {
        const int y = y0 + r, z = z0;
        for (int x = threadIdx.x; x < nx; x += blockDim.x) {
            const int cell = r * nx + x;                     // within the tile
            const R m0 = m0p[cell], m1 = m1p[cell], m2 = m2p[cell];
            const R ms = msarr ? msp[cell] : Msu;
            R H0 = 0, H1 = 0, H2 = 0, k0 = 0, k1 = 0, k2 = 0;
            if (ms > (R)0) {
                const R inv = msarr ? (R)1 / (mu0 * ms) : inv_u;
                R hd0 = 0, hd1 = 0, hd2 = 0;
                if (demag) {
                    const int pos = ix<true>(x >> 1, 1);
                    const V2<T> v0 = Hd[(3 * r + 0) * SK + pos];
                    const V2<T> v1 = Hd[(3 * r + 1) * SK + pos];
                    const V2<T> v2 = Hd[(3 * r + 2) * SK + pos];
                    hd0 = to_store<T>((x & 1) ? v0.y : v0.x);
                    hd1 = to_store<T>((x & 1) ? v1.y : v1.x);
                    hd2 = to_store<T>((x & 1) ? v2.y : v2.x);
                }
                // exchange (Eq. 5) and interfacial DMI (Eq. 14), free boundaries.  The six
                // neighbours are loaded unconditionally (a missing one reads the cell
                // itself) and masked afterwards, so all loads can be in flight together.
                R ex0 = 0, ex1 = 0, ex2 = 0, dm0 = 0, dm1 = 0, dm2 = 0;
                R gv[3] = {(R)0, (R)0, (R)0};                 // (u.grad)m, extended terms
                if (ext) {
                    R exv[3] = {(R)0, (R)0, (R)0}, dmv[3] = {(R)0, (R)0, (R)0};
                    ext_local<R>(d, cf, ext_coef<R>(d), m0p, m1p, m2p, msp, acp, dcp, cell, x, y, z, m0, m1, m2,
                                 inv, exv, dmv, gv);
                    ex0 = exv[0]; ex1 = exv[1]; ex2 = exv[2];
                    dm0 = dmv[0]; dm1 = dmv[1]; dm2 = dmv[2];
                } else if (do_ex || dmi) {
                    bool ok[6] = {x > 0, x < nx - 1, y > 0, y < ny - 1, z > 0, z < nz - 1};
                    const int off[6] = {-1, 1, -nx, nx, dzb, dza};
                    R j0[6], j1[6], j2[6];
#pragma unroll
                    for (int nb = 0; nb < 6; ++nb) {
                        const int o = cell + (ok[nb] ? off[nb] : 0);
                        j0[nb] = m0p[o]; j1[nb] = m1p[o]; j2[nb] = m2p[o];
                    }
                    if (msarr) {
                        const int moff[6] = {-1, 1, -nx, nx, -sz, sz};   // Ms stays in global memory
#pragma unroll
                        for (int nb = 0; nb < 6; ++nb) ok[nb] = ok[nb] && msp[cell + (ok[nb] ? moff[nb] : 0)] > (R)0;
                    }
                    if (do_ex) {
                        const R fe[6] = {ex_x, ex_x, ex_y, ex_y, ex_z, ex_z};
#pragma unroll
                        for (int nb = 0; nb < 6; ++nb) {
                            const R f = ok[nb] ? fe[nb] : (R)0;
                            ex0 += f * (j0[nb] - m0); ex1 += f * (j1[nb] - m1); ex2 += f * (j2[nb] - m2);
                        }
                        ex0 *= cA * inv; ex1 *= cA * inv; ex2 *= cA * inv;
                    }
                    if (dmi) {
                        // sum_j e_ij x m_j / Delta: -x:-e_y, +x:+e_y, -y:+e_x, +y:-e_x;
                        // e_y x m = (mz, 0, -mx), e_x x m = (0, -mz, my)
                        const R sxm = ok[0] ? -dm_x : (R)0, sxp = ok[1] ? dm_x : (R)0;
                        const R sym = ok[2] ? dm_y : (R)0, syp = ok[3] ? -dm_y : (R)0;
                        dm0 = sxm * j2[0] + sxp * j2[1];
                        dm2 = -(sxm * j0[0] + sxp * j0[1]) + sym * j1[2] + syp * j1[3];
                        dm1 = -(sym * j2[2] + syp * j2[3]);
                        dm0 *= -cD * inv; dm1 *= -cD * inv; dm2 *= -cD * inv;
                    }
                }
                R un0 = 0, un1 = 0, un2 = 0, cu0 = 0, cu1 = 0, cu2 = 0;
                if (do_uni) {
                    const R mu = m0 * ux + m1 * uy + m2 * uz;
                    const R f = cK * inv * mu;
                    un0 = f * ux; un1 = f * uy; un2 = f * uz;
                }
                if (do_cub) {
                    const R f = -cC * inv;
                    cu0 = f * m0 * m0 * m0; cu1 = f * m1 * m1 * m1; cu2 = f * m2 * m2 * m2;
                }
                H0 = hd0 + ex0 + dm0 + un0 + cu0 + Hx0;
                H1 = hd1 + ex1 + dm1 + un1 + cu1 + Hy0;
                H2 = hd2 + ex2 + dm2 + un2 + cu2 + Hz0;
                if (ENERGY) {
                    // per-cell densities in the context precision, accumulated per
                    // thread with FP64-level accuracy (CSum) and summed across
                    // threads in FP64; the constant factors are applied once per CTA
                    esum[0].add(ms * (m0 * ex0 + m1 * ex1 + m2 * ex2));
                    esum[1].add(ms * (m0 * dm0 + m1 * dm1 + m2 * dm2));
                    const R mu = m0 * ux + m1 * uy + m2 * uz;
                    esum[2].add(mu * mu);
                    const R q0 = m0 * m0, q1 = m1 * m1, q2 = m2 * m2;
                    esum[3].add(q0 * q0 + q1 * q1 + q2 * q2);
                    esum[4].add(ms * (m0 * Hx0 + m1 * Hy0 + m2 * Hz0));
                    esum[5].add(ms * (m0 * hd0 + m1 * hd1 + m2 * hd2));
                }
                // LL form: dm/dt = -g~ m x H - alpha g~ m x (m x H)
                const R c0 = m1 * H2 - m2 * H1, c1 = m2 * H0 - m0 * H2, c2 = m0 * H1 - m1 * H0;
                const R dd0 = m1 * c2 - m2 * c1, dd1 = m2 * c0 - m0 * c2, dd2 = m0 * c1 - m1 * c0;
                k0 = -agt * dd0; k1 = -agt * dd1; k2 = -agt * dd2;
                if (prec) { k0 -= gt * c0; k1 -= gt * c1; k2 -= gt * c2; }
                if (ext && (d.eflags & (E_STT | E_SOT))) ext_torque<R>(d, ext_coef<R>(d), m0, m1, m2, gv, k0, k1, k2);
            }
            const long long o = tile + cell;
            if (write_k) {
                p.kout[o] = k0; p.kout[o + N] = k1; p.kout[o + 2 * N] = k2;
            }
            if (p.heff) {
                p.heff[o] = H0; p.heff[o + N] = H1; p.heff[o + 2 * N] = H2;
            }
            if (red1) {
                // squared norm |dm/dt|^2 (a threshold / step-size estimate); the max
                // runs over ordered bits in the context precision, sqrt once per simulation
                vmax = umax64(vmax, obits(k0 * k0 + k1 * k1 + k2 * k2));
            } else if (red7) {
                // embedded error sum_j e_j k_j: e_1..e_6 part accumulated by the stage-7
                // prologue, plus e_7 k_7 in one correctly rounded FMA; h is applied
                // after the max (rounded scaling by h > 0 is monotone, so
                // max_i h|v_i| = h max_i |v_i| exactly)
                const R* ep = p.errp + o;
                vmax = umax64(vmax, obits(fabs(fma(e7, k0, ep[0]))));
                vmax = umax64(vmax, obits(fabs(fma(e7, k1, ep[N]))));
                vmax = umax64(vmax, obits(fabs(fma(e7, k2, ep[2 * N]))));
            }
        }
    }
    if (red1 || red7) {
        const unsigned long long rr = block_max_u64(vmax, red_u);
        if (threadIdx.x == 0) {
            // FP64 from here on: the CTA maximum, scaled by h at stage 7
            const double v = obits_to_double<R>(rr);
            const double vs = red7 ? fabs(p.state[w.sim].h * v) : v;
            atomicMax(red1 ? &p.state[w.sim].maxk_bits : &p.state[w.sim].err_bits,
                      (unsigned long long)__double_as_longlong(vs));
        }
    }
    if (ENERGY) {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int t = 0; t < 6; ++t) esum[t].warp_reduce();
        if (lane == 0) {
#pragma unroll
            for (int t = 0; t < 6; ++t) red_e[t * 32 + wid] = esum[t].value();
        }
        __syncthreads();
        if (threadIdx.x < 6) {
            // E_ex, E_dmi, E_d = -mu0/2 V sum Ms m.H;  E_zee = -mu0 V sum Ms m.H_ext;
            // E_uni = -Ku V sum (m.u)^2;  E_cub = Kc V sum (mx^4 + my^4 + mz^4)
            const double V = d.dx * d.dy * d.dz;
            const int t = threadIdx.x;
            const double scale = t == 2 ? -d.Ku * V : t == 3 ? d.Kc * V : t == 4 ? -kMu0 * V : -0.5 * kMu0 * V;
            double e = 0.0;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) e += red_e[t * 32 + i];
            atomicAdd(&p.state[w.sim].E[t], e * scale);
        }
    }
}

}  // namespace mm
