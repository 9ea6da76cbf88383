// Internal device-side definitions of libmm: simulation descriptors, kernel
// parameters, complex helpers and the in-place shared-memory FFT.
//
// Layouts (all simulations of a batch live in one set of buffers):
//   state  [3][nz][ny][nx] per simulation at element offset SimDesc::off
//   spectrum [3][nz][NBx][Py][Ty] complex per simulation at SimDesc::spec_off:
//          kx split into blocks of Ty columns so that a column tile is one
//          contiguous run; rows y < ny hold the x-transform, all Py rows the
//          xy-transform
//   tensor [ncomp][Pz/2+1][Py/2+1][Kx] real per geometry at SimDesc::tens_off,
//          ncomp = 6 (xx yy zz xy xz yz) or 4 when Pz == 1 (xz = yz = 0),
//          holding -N^(k)/(Px Py Pz); other bins follow from the parities
//          of the Newell tensor (diagonal even, xy odd in kx and ky, xz odd
//          in kx and kz, yz odd in ky and kz).  Films of the cluster-fused y/z
//          pass (2..8 planes) convolve along z directly and store the tensor
//          transformed along x and y only, blocked: [NBx][Py/2+1][Ty][yzc_qp(nz)],
//          entry 6 dz + c for dz = 0..nz-1 (-N^/(Px Py); xz and yz, odd in one of
//          x, y, are imaginary there and stored as their imaginary parts; negative
//          dz by the z parities), so one column's values for one ky are contiguous.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ddf.cuh"

#define MM_LOG2_LMAX 13
#define MM_LMAX (1 << MM_LOG2_LMAX)
#define MM_THREADS 256
// Cluster-fused y/z pass: largest plane count (portable cluster size) and its
// work lists, one per (planes, column group width, CTAs per SM):
// list = nz + kYzcLists * (wide + 2 occ), occ 0 for the rule's build, 1 for the
// one bounded for 3 CTAs per SM, 2 for 4 CTAs per SM.
constexpr int kMaxClusterPlanes = 8;
constexpr int kYzcLists = kMaxClusterPlanes + 1;
constexpr int kYzcListCount = 6 * kYzcLists;
// Plane counts with 3- and 4-CTA-per-SM builds of the FP32 cluster kernel.
constexpr int kYzcOcc3MaxPlanes = 4;
// Largest x-pass CTA (threads) per precision; as launch bounds with one CTA
// per SM it caps the x kernels at 64 (FP32) / 128 (FP64) registers a thread.
template <typename T>
constexpr int MM_XTHREADS_MAX = sizeof(T) == 4 ? 1024 : 512;

// Threads of an x- or column-pass CTA by the fixed rule.  Long rows and columns
// need large shared-memory tiles, which cap the CTAs resident on an SM (228 KB
// each); the CTA then widens so the SM still holds about `maxthreads` threads
// (the launch bound of those kernels).
inline int plan_wide_threads(size_t smem, int maxthreads) {
    int b = (int)(233472 / (smem + 1024));
    if (b < 1) b = 1;
    const int nt = 32 * ((maxthreads / b) / 32);
    return nt < MM_THREADS ? MM_THREADS : nt;
}

// F_DMI: interfacial DMI with D != 0; F_EX / F_UNI / F_CUB: A, Ku, Kc != 0.
// F_EXT: the simulation has extended terms (bulk or D_2d DMI, per-cell A / D,
// spin torques; SimDesc::eflags), evaluated by the extended x-inverse kernel;
// there F_DMI means DMI of the simulation's class with a non-zero constant and
// F_EX exchange with a non-zero uniform or per-cell constant.
// F_XSTAGE: the x-inverse pass stages the tile's state rows (with their +-y and
// +-z neighbours) into shared memory by bulk copies (the planner reserved room).
enum { F_DEMAG = 1, F_DMI = 2, F_PREC = 4, F_MSARR = 8, F_EX = 16, F_UNI = 32, F_CUB = 64, F_EXT = 128,
       F_XSTAGE = 256 };
// extended terms: per-cell A and D, Zhang-Li torque, Slonczewski / spin-orbit torque
enum { E_CELL = 1, E_STT = 2, E_SOT = 4 };

// Coefficients of the local fields and of the LL torque of one simulation in
// one precision, computed once on the host (plan_coefficients).  GB300 runs
// FP64 at a small fraction of its FP32 rate, so the kernels of an FP32
// context read these instead of dividing and converting FP64 material
// parameters in every thread.
template <typename T>
struct Coef {
    T Ms;                // uniform saturation magnetisation
    T mu0;
    T inv_u;             // 1 / (mu0 Ms) for uniform Ms (0 when Ms = 0)
    T ex[3];             // 1/dx^2, 1/dy^2, 1/dz^2
    T dm[2];             // 1/dx, 1/dy
    T cA, cD, cK, cC;    // 2A, D, 2Ku, 4Kc
    T u[3], H[3];
    T gt, agt;           // gamma/(1+alpha^2), alpha gamma/(1+alpha^2)
    T pad;
};

// Coefficients of the extended terms in one precision (plan_extended).
template <typename T>
struct ExtCoef {
    T A, D;              // uniform exchange and DMI constants
    T dinv_z;            // 1/dz (DMI along z)
    T gu[3];             // u_c / (2 Delta_c): central-difference (u.grad)m
    T beta, aJ, bJ;      // non-adiabaticity, Slonczewski / spin-orbit strengths (1/s)
    T alpha, inv_q;      // alpha, 1 / (1 + alpha^2)
    T p[3];              // unit polarisation
};

struct SimDesc {
    int nx, ny, nz, ncells;
    int Px, Py, Pz;
    int lPx, lPy, lPz;       // log2 of the padded sizes
    int Kx;                  // Px/2 + 1
    int Pyh, Pzh;            // tensor bins along y and z
    int ncomp;               // 4 or 6
    int flags;
    int Rx;                  // rows per CTA in the x passes
    int Ty;                  // kx block width (power of two): spectrum block and column tile
    int lTy;                 // log2(Ty)
    int NBx;                 // number of kx blocks, ceil(Kx / Ty)
    int group_begin, group_end;   // NEB chain members [begin, end), -1 if none
    int neb_index;                // image index in its chain
    int colgroup;                 // cluster-pass column register groups: 0 rule, 1 16-point, 2 32-point
    int yzcocc;                   // cluster-pass CTAs per SM the kernel is compiled for: 0 rule (2), 3, 4
    int pad0;
    long long off;           // element offset of the [3][N] state block
    long long spec_off;      // complex offset of the spectrum block
    long long ms_off;        // offset into the per-cell Ms array, -1 if uniform
    long long tens_off;      // element offset of the tensor block
    double Ms, A, D, Ku, u[3], Kc, H[3], alpha, gamma;
    double dx, dy, dz;
    double k_spring;
    Coef<double> cd;         // the coefficients in FP64 and in FP32
    Coef<float> cf;
    int dmi_kind;            // 0 none, 1 interfacial, 2 bulk, 3 D_2d
    int eflags;              // E_CELL | E_STT | E_SOT
    long long cell_off;      // per-cell [A][D] block (2 ncells values), -1 if none
    double u_stt[3], beta, aJ, bJ, p[3];
    ExtCoef<double> xd;      // extended-term coefficients in FP64 and in FP32
    ExtCoef<float> xf;
};

template <typename T> __host__ __device__ __forceinline__ const Coef<T>& coef(const SimDesc& d);
template <> __host__ __device__ __forceinline__ const Coef<double>& coef<double>(const SimDesc& d) { return d.cd; }
template <> __host__ __device__ __forceinline__ const Coef<float>& coef<float>(const SimDesc& d) { return d.cf; }
template <typename T> __host__ __device__ __forceinline__ const ExtCoef<T>& ext_coef(const SimDesc& d);
template <> __host__ __device__ __forceinline__ const ExtCoef<double>& ext_coef<double>(const SimDesc& d) { return d.xd; }
template <> __host__ __device__ __forceinline__ const ExtCoef<float>& ext_coef<float>(const SimDesc& d) { return d.xf; }

struct SimState {
    double t, h, t_end, rtol, max_dmdt;
    double err, maxk;
    unsigned long long err_bits;     // max of |h sum e_j k_j| as ordered bits (NaN wins)
    unsigned long long maxk_bits;    // max |dm/dt|^2 over cells at stage 1 (ordered bits)
    long long n_acc, n_rej;
    int status, accepted, pad1, pad2;
    double E[8];                     // energy accumulators (ex, dmi, uni, cub, zee, demag)
    double neb[4];                   // NEB reductions: |tau|^2, H.tau, distance to next image
};

struct WorkItem { int sim, a, b, c; };

// Tensor values per (kx, ky) bin in the blocked layout of the cluster-fused
// y/z pass: the 6 components at the dz = 0..nz-1 plane offsets, padded to a
// multiple of 4 for 16-byte vector loads.
__host__ __device__ constexpr int yzc_qp(int nz) { return ((6 * nz + 3) / 4) * 4; }

template <typename T> struct alignas(2 * sizeof(T)) V2 { T x, y; };

template <typename T> __device__ __forceinline__ V2<T> mk(T x, T y) { V2<T> r; r.x = x; r.y = y; return r; }
template <typename T> __device__ __forceinline__ V2<T> operator+(V2<T> a, V2<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ V2<T> operator-(V2<T> a, V2<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ V2<T> cmul(V2<T> a, V2<T> b) {
    return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __device__ __forceinline__ V2<T> cconj(V2<T> a) { return mk<T>(a.x, -a.y); }
template <typename T> __device__ __forceinline__ V2<T> cscale(V2<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <typename T, bool INV> __device__ __forceinline__ V2<T> mul_mi(V2<T> a) {
    return INV ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
}

__device__ __forceinline__ int bitrev(int v, int bits) {
    return bits == 0 ? 0 : (int)(__brev((unsigned)v) >> (32 - bits));
}

// twiddle W_M^k = exp(-+2 pi i k / M), M = 2^logM, from the table of exp(-2 pi i j / LMAX)
template <typename T, bool INV>
__device__ __forceinline__ V2<T> twid(const V2<T>* __restrict__ tw, int k, int logM) {
    V2<T> w = tw[k << (MM_LOG2_LMAX - logM)];
    if (INV) w.y = -w.y;
    return w;
}

// Stage twiddle tables, stored after the MM_LMAX-entry table: for radix
// R = 2^LR (LR = 1..4) and length M = 2^lM (LR <= lM <= MM_LOG2_LMAX), the
// values W_M^(k r) for r = 1..R-1 and k < M/R at stw_base(LR, lM) + (r-1) M/R + k.
// Consecutive k are adjacent, so the butterflies of a warp read one contiguous
// run per r (the MM_LMAX table, read at stride LMAX/M, puts every lane of a
// warp on its own sector).  (LR = 1, lM) is W_M^k for k < M/2.
__host__ __device__ constexpr int stw_size(int LR) { return ((1 << LR) - 1) * ((1 << (MM_LOG2_LMAX + 1 - LR)) - 1); }
__host__ __device__ constexpr int stw_off(int LR) { return LR <= 1 ? 0 : stw_off(LR - 1) + stw_size(LR - 1); }
__host__ __device__ constexpr int stw_base(int LR, int lM) { return stw_off(LR) + ((1 << LR) - 1) * ((1 << (lM - LR)) - 1); }
#define MM_STW_ENTRIES (stw_off(5))
#define MM_TW_ENTRIES (MM_LMAX + MM_STW_ENTRIES)

template <typename T, bool INV>
__device__ __forceinline__ V2<T> stw_get(const V2<T>* __restrict__ t, int i) {
    V2<T> w = t[i];
    if (INV) w.y = -w.y;
    return w;
}

// Map a linear butterfly index to (sequence, group).  Sequences stored with
// unit element stride are walked group-fastest; interleaved sequences
// (element stride > 1) sequence-fastest, so a warp touches adjacent words.
__device__ __forceinline__ void split_id(int id, int ngroups, int nseq, int estride, int& seq, int& g) {
    if (estride == 1) { seq = id / ngroups; g = id - seq * ngroups; }
    else { g = id / nseq; seq = id - g * nseq; }
}

// Element j of a unit-stride sequence sits at pidx(j) = j + j/16: one pad
// slot per 16 complex values keeps the radix-4 access patterns off shared
// memory bank conflicts.  Padded length of an n-element sequence:
__host__ __device__ __forceinline__ int padded_len(int n) { return n + (n >> 4) + 1; }

template <bool PAD>
__device__ __forceinline__ int ix(int j, int estride) { return PAD ? j + (j >> 4) : j * estride; }

// Length-PZ FFT of one sequence held in registers (PZ = 2, 4, 8, 16), natural
// order in and out; radix-2 decimation in time, unnormalised.
template <int PZ> struct Log2 { static constexpr int v = PZ == 2 ? 1 : PZ == 4 ? 2 : PZ == 8 ? 3 : 4; };

template <int BITS>
__host__ __device__ constexpr int brev_ct(int v) {
    int r = 0;
    for (int i = 0; i < BITS; ++i) r |= ((v >> i) & 1) << (BITS - 1 - i);
    return r;
}

// cos(2 pi k / 32), k = 0..7 (the rest of the circle by symmetry)
__device__ __forceinline__ double w32c(int k) {
    return k == 0 ? 1.0
         : k == 1 ? 0.9807852804032304491261822
         : k == 2 ? 0.9238795325112867561281832
         : k == 3 ? 0.8314696123025452370787884
         : k == 4 ? 0.7071067811865475244008444
         : k == 5 ? 0.5555702330196022247428308
         : k == 6 ? 0.3826834323650897717284600
         : 0.1950903220161282678482849;
}

// W_M^r = exp(-+2 pi i r / M) for M <= 32, from compile-time constants
template <typename T, bool INV>
__device__ __forceinline__ V2<T> small_twid(int r, int logM) {
    const int q = r << (5 - logM);              // in 32nds of a turn, 0..31
    const int qm = q & 7;
    const T c = (T)w32c(qm);                    // cos and sin of qm/32 turn
    const T sn = qm == 0 ? (T)0 : (T)w32c(8 - qm);
    // rotate by the quarter turns in q >> 3: (c, -sn) * (-i)^(q>>3)
    V2<T> w;
    switch (q >> 3) {
        case 0: w = mk<T>(c, -sn); break;
        case 1: w = mk<T>(-sn, -c); break;
        case 2: w = mk<T>(-c, sn); break;
        default: w = mk<T>(sn, c); break;
    }
    if (INV) w.y = -w.y;
    return w;
}

// a * (-i)^m (forward) or (+i)^m (INV): swaps and sign flips only
template <typename T, bool INV>
__device__ __forceinline__ V2<T> rot_quarter(V2<T> a, int m) {
    switch (m & 3) {
        case 0: return a;
        case 1: return INV ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
        case 2: return mk<T>(-a.x, -a.y);
        default: return INV ? mk<T>(a.y, -a.x) : mk<T>(-a.y, a.x);
    }
}

// a * W_32^q (INV: conjugate) for q fixed at compile time after unrolling:
// quarter turns cost no arithmetic, odd eighth turns two adds and two
// multiplies by sqrt(1/2), the rest a full complex product.  (IEEE rules keep
// the compiler from folding the zero and unit parts of a general product, and
// FP64 arithmetic is scarce on GB300.)
template <typename T, bool INV>
__device__ __forceinline__ V2<T> cmul_tw32(V2<T> a, int q) {
    q &= 31;
    if ((q & 7) == 0) return rot_quarter<T, INV>(a, q >> 3);
    if ((q & 3) == 0) {
        const T h = (T)0.7071067811865475244008444;
        const V2<T> b = INV ? mk<T>(h * (a.x - a.y), h * (a.x + a.y)) : mk<T>(h * (a.x + a.y), h * (a.y - a.x));
        return rot_quarter<T, INV>(b, q >> 3);
    }
    return cmul(a, small_twid<T, INV>(q, 5));
}

template <typename T, int PZ, bool INV>
__device__ __forceinline__ void reg_fft(V2<T> (&x)[PZ], const V2<T>* __restrict__ tw) {
    constexpr int LG = Log2<PZ>::v;
    V2<T> y[PZ];
#pragma unroll
    for (int i = 0; i < PZ; ++i) y[brev_ct<LG>(i)] = x[i];
#pragma unroll
    for (int lg = 0; lg < LG; ++lg) {
        const int s = 1 << lg;
#pragma unroll
        for (int base = 0; base < PZ; base += 2 * s) {
#pragma unroll
            for (int r = 0; r < s; ++r) {
                // W_{2s}^r = W_32^(r 32 / 2s)
                const V2<T> a = y[base + r], b = cmul_tw32<T, INV>(y[base + r + s], r << (4 - lg));
                y[base + r] = a + b;
                y[base + r + s] = a - b;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < PZ; ++i) x[i] = y[i];
}

// One Stockham auto-sort stage of radix R over nseq padded (pidx) sequences of
// length 2^lL, from src to dst: butterfly j reads x[j + r L/R], multiplies by
// W_{Ns R}^{(j mod Ns) r}, does an R-point DFT in registers and writes
// x'[(j / Ns) Ns R + (j mod Ns) + r Ns], Ns = 2^lNs the length already
// transformed.  Natural order in, natural order out after the last stage.
// ZIN (first stage only): the upper half of the input is zero and is not read.
// HOUT (last stage only): only the lower half of the output is written.
// tw points at the MM_LMAX table; the stage tables follow it.
template <typename T, bool INV, int R, bool ZIN, bool HOUT>
__device__ __forceinline__ void stockham_stage(const V2<T>* src, V2<T>* dst, int lL, int lNs, int nseq, int sstride,
                                               const V2<T>* __restrict__ tw) {
    constexpr int LR = Log2<R>::v;
    const int lnb = lL - LR;
    const int nb = 1 << lnb;
    const int tot = nseq << lnb;
    const V2<T>* __restrict__ st = tw + MM_LMAX + stw_base(LR, lNs + LR);
    for (int id = threadIdx.x; id < tot; id += blockDim.x) {
        const int seq = id >> lnb, j = id & (nb - 1);
        const V2<T>* s = src + seq * sstride;
        V2<T>* d = dst + seq * sstride;
        const int k = j & ((1 << lNs) - 1);
        V2<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r)
            v[r] = (ZIN && r >= R / 2) ? mk<T>((T)0, (T)0) : s[ix<true>(j + (r << lnb), 1)];
        if (!ZIN && lNs > 0) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], stw_get<T, INV>(st, ((r - 1) << lNs) + k));
        }
        reg_fft<T, R, INV>(v, tw);
        const int o = ((j >> lNs) << (lNs + LR)) + k;
#pragma unroll
        for (int r = 0; r < (HOUT ? R / 2 : R); ++r) d[ix<true>(o + (r << lNs), 1)] = v[r];
    }
}

template <typename T, bool INV, int R, bool ZIN, bool HOUT>
__device__ __forceinline__ void stockham_pick(const V2<T>* a, V2<T>* b, int lL, int lNs, int nseq, int sstride,
                                              const V2<T>* __restrict__ tw, bool first, bool last) {
    if (ZIN && first) {
        if (HOUT && last) stockham_stage<T, INV, R, true, true>(a, b, lL, lNs, nseq, sstride, tw);
        else stockham_stage<T, INV, R, true, false>(a, b, lL, lNs, nseq, sstride, tw);
    } else {
        if (HOUT && last) stockham_stage<T, INV, R, false, true>(a, b, lL, lNs, nseq, sstride, tw);
        else stockham_stage<T, INV, R, false, false>(a, b, lL, lNs, nseq, sstride, tw);
    }
}

// Full unnormalised FFT of nseq padded sequences of length 2^lL (natural
// order in and out) with Stockham stages of radix up to 2^MAXLR, ping-ponging
// between a and b.  Returns the buffer that holds the result.  Ends with
// __syncthreads().  ZIN: the upper half of every input sequence is zero (it
// need not be stored); HOUT: only the lower half of the result is wanted
// (the upper half is left undefined).
template <typename T, bool INV, int MAXLR, bool ZIN = false, bool HOUT = false>
__device__ V2<T>* stockham_fft(V2<T>* a, V2<T>* b, int lL, int nseq, int sstride, const V2<T>* __restrict__ tw) {
    int lNs = 0;
    while (lNs < lL) {
        const int rem = lL - lNs;
        int lr = rem < MAXLR ? rem : MAXLR;
        if (rem - lr == 1 && lr > 2) lr -= 1;          // avoid a trailing radix-2 stage
        const bool first = lNs == 0, last = lNs + lr == lL;
        switch (lr) {
            case 1: stockham_pick<T, INV, 2, ZIN, HOUT>(a, b, lL, lNs, nseq, sstride, tw, first, last); break;
            case 2: stockham_pick<T, INV, 4, ZIN, HOUT>(a, b, lL, lNs, nseq, sstride, tw, first, last); break;
            case 3: stockham_pick<T, INV, 8, ZIN, HOUT>(a, b, lL, lNs, nseq, sstride, tw, first, last); break;
            default:
                stockham_pick<T, INV, (MAXLR >= 4 ? 16 : 8), ZIN, HOUT>(a, b, lL, lNs, nseq, sstride, tw, first,
                                                                      last);
                break;
        }
        __syncthreads();
        V2<T>* t = a; a = b; b = t;
        lNs += lr;
    }
    return a;
}

// In-place radix-2 FFT stages processed in groups of G consecutive stages: a
// work item loads the 2^G elements base + r + m s (m < 2^G) of one block,
// runs the G butterfly stages in registers, and stores them back, so a
// group costs one shared-memory round trip and one barrier.  The twiddle of
// stage t for offset u = m mod 2^t is W_{s 2^(t+1)}^r * W_{2^(t+1)}^u (table
// times compile-time constant).  Checked against numpy's FFT for lengths
// 1..1024 and every group size.
// HOUT (last group only): only the lower half of the sequence is wanted; the
// last stage skips its differences and the upper half is not stored.
template <typename T, bool INV, int G, bool PAD, bool HOUT = false>
__device__ __forceinline__ void dit_group(V2<T>* buf, int lL, int lg, int nseq, int sstride, int estride,
                                          const V2<T>* __restrict__ tw) {
    constexpr int M = 1 << G;
    const int ng = 1 << (lL - G);
    const int tot = ng * nseq;
    const int s = 1 << lg;
    for (int id = threadIdx.x; id < tot; id += blockDim.x) {
        int seq, g;
        split_id(id, ng, nseq, estride, seq, g);
        V2<T>* p = buf + seq * sstride;
        const int r = g & (s - 1);
        const int base = ((g >> lg) << (lg + G)) + r;
        V2<T> v[M];
#pragma unroll
        for (int m = 0; m < M; ++m) v[m] = p[ix<PAD>(base + m * s, estride)];
#pragma unroll
        for (int t = 0; t < G; ++t) {
            const int h = 1 << t;
            const V2<T> wb = twid<T, INV>(tw, r, lg + t + 1);
#pragma unroll
            for (int m = 0; m < M; ++m) {
                if (m & h) continue;
                const int u = m & (h - 1);
                const V2<T> w = u ? cmul_tw32<T, INV>(wb, u << (4 - t)) : wb;   // wb W_{2^(t+1)}^u
                const V2<T> a = v[m], b = cmul(v[m + h], w);
                v[m] = a + b;
                if (!(HOUT && t == G - 1)) v[m + h] = a - b;
            }
        }
#pragma unroll
        for (int m = 0; m < (HOUT ? M / 2 : M); ++m) p[ix<PAD>(base + m * s, estride)] = v[m];
    }
}

// ZIN (first group only): the upper half of the sequence is zero; it is not
// read and the first stage reduces to v[m + M/2] = v[m] w.
template <typename T, bool INV, int G, bool PAD, bool ZIN = false>
__device__ __forceinline__ void dif_group(V2<T>* buf, int lL, int lS, int nseq, int sstride, int estride,
                                          const V2<T>* __restrict__ tw) {
    constexpr int M = 1 << G;
    const int ng = 1 << (lL - G);
    const int tot = ng * nseq;
    const int lsm = lS - G + 1;                  // smallest span of the group
    const int sm = 1 << lsm;
    for (int id = threadIdx.x; id < tot; id += blockDim.x) {
        int seq, g;
        split_id(id, ng, nseq, estride, seq, g);
        V2<T>* p = buf + seq * sstride;
        const int r = g & (sm - 1);
        const int base = ((g >> lsm) << (lS + 1)) + r;
        V2<T> v[M];
#pragma unroll
        for (int m = 0; m < M; ++m) v[m] = (ZIN && m >= M / 2) ? mk<T>((T)0, (T)0) : p[ix<PAD>(base + m * sm, estride)];
#pragma unroll
        for (int t = G - 1; t >= 0; --t) {
            const int h = 1 << t;
            const V2<T> wb = twid<T, INV>(tw, r, lsm + t + 1);
#pragma unroll
            for (int m = 0; m < M; ++m) {
                if (m & h) continue;
                const int u = m & (h - 1);
                const V2<T> w = u ? cmul_tw32<T, INV>(wb, u << (4 - t)) : wb;   // wb W_{2^(t+1)}^u
                if (ZIN && t == G - 1) {
                    v[m + h] = cmul(v[m], w);        // b = 0: a + b = a, (a - b) w = a w
                } else {
                    const V2<T> a = v[m], b = v[m + h];
                    v[m] = a + b;
                    v[m + h] = cmul(a - b, w);
                }
            }
        }
#pragma unroll
        for (int m = 0; m < M; ++m) p[ix<PAD>(base + m * sm, estride)] = v[m];
    }
}

// Stages per register group: logL stages in ceil(logL / GM) groups of
// near-equal size (a trailing group of one or two stages costs almost as
// much per element as a full one).  Group i of the schedule:
__device__ __forceinline__ int group_size(int logL, int GM, int i) {
    const int ng = (logL + GM - 1) / GM;
    const int b = logL / ng;
    return b + (i < logL - b * ng ? 1 : 0);
}

template <typename T, bool INV, int G, bool PAD, bool HOUT>
__device__ __forceinline__ void dit_pick(V2<T>* buf, int logL, int lg, int nseq, int sstride, int estride,
                                         const V2<T>* __restrict__ tw, bool last) {
    if (HOUT && last) dit_group<T, INV, G, PAD, true>(buf, logL, lg, nseq, sstride, estride, tw);
    else dit_group<T, INV, G, PAD, false>(buf, logL, lg, nseq, sstride, estride, tw);
}

template <typename T, bool INV, int G, bool PAD, bool ZIN>
__device__ __forceinline__ void dif_pick(V2<T>* buf, int logL, int lS, int nseq, int sstride, int estride,
                                         const V2<T>* __restrict__ tw, bool first) {
    if (ZIN && first) dif_group<T, INV, G, PAD, true>(buf, logL, lS, nseq, sstride, estride, tw);
    else dif_group<T, INV, G, PAD, false>(buf, logL, lS, nseq, sstride, estride, tw);
}

// Default largest group: 16 points (FP32) / 8 (FP64) in registers; kernels
// with a larger register budget pass GM = 5.
template <typename T>
constexpr int kGroupMax = sizeof(T) == 4 ? 4 : 3;

// In-place decimation-in-time FFT of nseq sequences of length 2^logL held in
// shared memory in BIT-REVERSED order; leaves them in natural order.
// Unnormalised.  Ends with __syncthreads().  PAD: unit-stride sequences
// stored with pidx() padding (estride ignored).  HOUT: only the lower half of
// each result is wanted (the upper half is left undefined).  GM: largest
// group (log2 of the points held in registers).
template <typename T, bool INV, bool PAD = false, bool HOUT = false, int GM = kGroupMax<T>>
__device__ void fft_dit(V2<T>* buf, int logL, int nseq, int sstride, int estride,
                        const V2<T>* __restrict__ tw) {
    int lg = 0;
    for (int i = 0; lg < logL; ++i) {
        const int G = group_size(logL, GM, i);
        const bool last = lg + G == logL;
        switch (G) {
            case 1: dit_pick<T, INV, 1, PAD, HOUT>(buf, logL, lg, nseq, sstride, estride, tw, last); break;
            case 2: dit_pick<T, INV, 2, PAD, HOUT>(buf, logL, lg, nseq, sstride, estride, tw, last); break;
            case 3: dit_pick<T, INV, 3, PAD, HOUT>(buf, logL, lg, nseq, sstride, estride, tw, last); break;
            case 4:
                if constexpr (GM >= 4) dit_pick<T, INV, 4, PAD, HOUT>(buf, logL, lg, nseq, sstride, estride, tw, last);
                break;
            default:
                if constexpr (GM >= 5) dit_pick<T, INV, 5, PAD, HOUT>(buf, logL, lg, nseq, sstride, estride, tw, last);
                break;
        }
        __syncthreads();
        lg += G;
    }
}

// In-place decimation-in-frequency FFT: natural order in, BIT-REVERSED order
// out.  Unnormalised.  Ends with __syncthreads().  ZIN: the upper half of each
// input is zero (it need not be stored).  GM as for fft_dit.
template <typename T, bool INV, bool PAD = false, bool ZIN = false, int GM = kGroupMax<T>>
__device__ void fft_dif(V2<T>* buf, int logL, int nseq, int sstride, int estride,
                        const V2<T>* __restrict__ tw) {
    int lS = logL - 1;
    for (int i = 0; lS >= 0; ++i) {
        const int G = group_size(logL, GM, i);
        const bool first = i == 0;
        switch (G) {
            case 1: dif_pick<T, INV, 1, PAD, ZIN>(buf, logL, lS, nseq, sstride, estride, tw, first); break;
            case 2: dif_pick<T, INV, 2, PAD, ZIN>(buf, logL, lS, nseq, sstride, estride, tw, first); break;
            case 3: dif_pick<T, INV, 3, PAD, ZIN>(buf, logL, lS, nseq, sstride, estride, tw, first); break;
            case 4:
                if constexpr (GM >= 4) dif_pick<T, INV, 4, PAD, ZIN>(buf, logL, lS, nseq, sstride, estride, tw, first);
                break;
            default:
                if constexpr (GM >= 5) dif_pick<T, INV, 5, PAD, ZIN>(buf, logL, lS, nseq, sstride, estride, tw, first);
                break;
        }
        __syncthreads();
        lS -= G;
    }
}

// Dormand & Prince (1980) RK5(4)7M: a_{s,j} (stage s = 2..7, j = 0..s-2) and the
// error weights e_j = b_j - bhat_j (j = 0..6).  constexpr so that stage kernels
// fold them (and skip the zero ones) at compile time.
__host__ __device__ constexpr double dp_a(int s, int j) {
    return s == 2 ? (j == 0 ? 1.0 / 5 : 0.0)
         : s == 3 ? (j == 0 ? 3.0 / 40 : j == 1 ? 9.0 / 40 : 0.0)
         : s == 4 ? (j == 0 ? 44.0 / 45 : j == 1 ? -56.0 / 15 : j == 2 ? 32.0 / 9 : 0.0)
         : s == 5 ? (j == 0 ? 19372.0 / 6561 : j == 1 ? -25360.0 / 2187 : j == 2 ? 64448.0 / 6561
                    : j == 3 ? -212.0 / 729 : 0.0)
         : s == 6 ? (j == 0 ? 9017.0 / 3168 : j == 1 ? -355.0 / 33 : j == 2 ? 46732.0 / 5247
                    : j == 3 ? 49.0 / 176 : j == 4 ? -5103.0 / 18656 : 0.0)
         : s == 7 ? (j == 0 ? 35.0 / 384 : j == 1 ? 0.0 : j == 2 ? 500.0 / 1113 : j == 3 ? 125.0 / 192
                    : j == 4 ? -2187.0 / 6784 : j == 5 ? 11.0 / 84 : 0.0)
         : 0.0;
}
__host__ __device__ constexpr double dp_e(int j) {
    return j == 0 ? 71.0 / 57600 : j == 1 ? 0.0 : j == 2 ? -71.0 / 16695 : j == 3 ? 71.0 / 1920
         : j == 4 ? -17253.0 / 339200 : j == 5 ? 22.0 / 525 : j == 6 ? -1.0 / 40 : 0.0;
}

// Parameters of every pass kernel (passed by value).
enum { MODE_RHS = 0, MODE_RK = 1, MODE_ENERGY = 2, MODE_NEB = 3 };

// T: the type the transforms compute in (float, double, or dd for FP64
// contexts); S = StoreT<T>: the type of the state, stage vectors, fields, Ms and
// per-cell constants in memory (float or double).  The spectrum, tensor and
// twiddles are stored in T.
template <typename T>
struct PassParams {
    using S = StoreT<T>;
    const SimDesc* __restrict__ desc;
    SimState* state;
    const WorkItem* __restrict__ items;
    int mode;
    int stage;              // 1..7 in MODE_RK
    int nk;                 // number of k vectors combined by the RK prologue
    int write_y;            // prologue writes the stage state
    double a[7];            // RK coefficients a_{s,j}
    double e[7];            // error coefficients (stage 7)
    const S* m;             // y_n (MODE_RK) or the evaluated state (other modes)
    S* ybuf;                // stage state
    S* const* kvec;         // k_1..k_7 (device array of 7 pointers)
    S* kout;                // k_s / dm/dt output
    S* heff;                // optional H_eff output
    S* errp;                // partial error vector (stage 7)
    long long off_adjust;   // subtracted from SimDesc::off for caller buffers of one simulation
    V2<T>* spec;
    const T* __restrict__ tensor;
    const S* __restrict__ Ms;
    const V2<T>* __restrict__ tw;
    const S* __restrict__ cellp;   // per-cell A and D blocks (SimDesc::cell_off)
};

// Asynchronous 16-byte global -> shared copies (cp.async, L2 only): a CTA
// issues all its tile loads without holding them in registers, then waits for
// its own copies once.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Staged state rows of the x-inverse pass (F_XSTAGE): after its two FFT buffers
// (nseq padded sequences of SK complex values each, vsz bytes a value), rounded up
// to 16 bytes, the three components' rows y0-1 .. y0+nrows (those in the mesh),
// then the nrows rows of the plane below and of the plane above, esz bytes a value.
__host__ __device__ constexpr size_t xinv_stage_offset(int nseq, int SK, size_t vsz) {
    return ((2 * (size_t)nseq * SK * vsz) + 15) & ~(size_t)15;
}
__host__ __device__ constexpr size_t xinv_stage_bytes(int nrows, int nx, size_t esz) {
    return 3 * (size_t)(3 * nrows + 2) * nx * esz;
}

// Bulk copies (the copy engine of sm_90+, cp.async.bulk) of contiguous global
// ranges into shared memory, completed on an mbarrier by transaction count.
// Addresses 16-byte aligned, sizes multiples of 16 bytes.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* smem_dst, const void* gmem_src, unsigned bytes,
                                         unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(smem_dst)),
        "l"(gmem_src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// One bounded probe of the barrier's phase; true once phase `parity` has completed.
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for phase `parity` with at most `limit` probes; false if it ran out.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity, int limit) {
    for (int i = 0; i < limit; ++i)
        if (mbar_test(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ double bits_to_double(unsigned long long b) { return __longlong_as_double((long long)b); }

// Ordered bits of a non-negative value in the context precision: for v >= 0
// (and NaN, which compares above +inf) integer order is value order, so a max
// over bits is exact and lets a NaN win.  obits_to_double converts a maximum
// back to FP64 once per CTA.
__device__ __forceinline__ unsigned long long obits(float v) { return (unsigned long long)__float_as_uint(v); }
__device__ __forceinline__ unsigned long long obits(double v) { return (unsigned long long)__double_as_longlong(v); }
template <typename T> __device__ __forceinline__ double obits_to_double(unsigned long long b);
template <> __device__ __forceinline__ double obits_to_double<float>(unsigned long long b) {
    return (double)__uint_as_float((unsigned)b);
}
template <> __device__ __forceinline__ double obits_to_double<double>(unsigned long long b) {
    return __longlong_as_double((long long)b);
}

// Error-free transformations (Knuth's TwoSum, Dekker's product through an
// FMA): a + b = s + e and a * b = p + e exactly in binary floating point.
// The _rn intrinsics keep the compiler from contracting or reordering them.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// Per-thread sum with FP64-level accuracy: an FP32 context accumulates a
// compensated (float-float) sum with FP32 operations, an FP64 context a plain
// FP64 sum; value() is the FP64 total handed to the FP64 block reduction.
template <typename T> struct CSum;
template <> struct CSum<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        float t, e;
        two_sum(s, v, t, e);
        s = t;
        c = __fadd_rn(c, e);
    }
    // sum over the warp (float-float additions), result in every lane
    __device__ __forceinline__ void warp_reduce() {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float so = __shfl_xor_sync(0xffffffffu, s, o), co = __shfl_xor_sync(0xffffffffu, c, o);
            float t, e;
            two_sum(s, so, t, e);
            s = t;
            c = __fadd_rn(__fadd_rn(c, co), e);
        }
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};
template <> struct CSum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ void warp_reduce() {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    __device__ __forceinline__ double value() const { return s; }
};
