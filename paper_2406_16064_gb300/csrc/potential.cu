// Demagnetising field through the magnetic scalar potential: three forward
// transforms and one inverse (Sec. "Magnetostatic energy": with the scalar
// potential the three inverse transforms of the FFT demag reduce to one).
//
//   u_i = sum_j S(r_i - r_j) . M_j,   H_d = -grad u   (central differences)
//
// S_c(R) is the exact potential at offset R of one cell magnetised with unit
// magnetisation along c: the cell's two c-faces carry surface charge +-1, so
// S_x(R) = (1/4 pi) [P(X - dx/2; Y, Z) - P(X + dx/2; Y, Z)] with P(a; Y, Z) the
// potential of a uniformly charged dy x dz rectangle at normal distance a,
// from the mixed antiderivative F(y, z) = y ln(z + r) + z ln(y + r) -
// a atan(y z / (a r)) of 1/r at its four corners (S_y, S_z by permuting the
// axes).  The potential is needed one cell outside the mesh on each side of
// every axis (the central difference at a boundary cell), so the convolution
// is taken on a grid padded to a power of two P >= 2n + 1 per axis (offsets
// -n..n), and the inverse transform keeps the n + 2 positions -1..n of each axis.
//
// Passes (one launch each, T = float or double; the tensor in FP64):
//   k_pot_sx      S_c on one padded row, complex FFT along x -> bins 0..Px/2
//   k_pot_mx      M = Ms m on one mesh row, zero-padded FFT along x -> bins 0..Px/2
//   k_pot_col     FFT along y or z of tiles of kx columns (forward or inverse)
//   k_pot_dot     u^ = sum_c S^_c M^_c per bin (S^ scaled by 1 / (Px Py Pz))
//   k_pot_xinv    Hermitian completion and inverse FFT along x of one output row,
//                 positions -1..nx kept
//   k_pot_grad    H_d = -grad u by central differences at every cell
#include <cmath>

#include "mm_kernels.cuh"
#include "potential.h"

namespace mm {

namespace {

constexpr double kPiP = 3.14159265358979323846;

// ln(z + r) with r = sqrt(z^2 + rest2), rest2 > 0; for z < 0 through z + r = rest2 / (r - z)
__device__ double pot_log_sum(double z, double r, double rest2) {
    return z >= 0.0 ? log(z + r) : log(rest2) - log(r - z);
}

// F(y, z) with d^2 F / (dy dz) = 1 / sqrt(a^2 + y^2 + z^2), a != 0
__device__ double pot_corner(double a, double y, double z) {
    const double r = sqrt(a * a + y * y + z * z);
    double v = 0.0;
    if (y != 0.0) v += y * pot_log_sum(z, r, a * a + y * y);
    if (z != 0.0) v += z * pot_log_sum(y, r, a * a + z * z);
    return v - a * atan(y * z / (a * r));
}

// integral of 1 / |r - s| over the rectangle [Y - dy/2, Y + dy/2] x [Z - dz/2, Z + dz/2]
// of the plane at normal distance a from r
__device__ double pot_rect(double a, double Y, double Z, double dy, double dz) {
    const double y1 = -Y - 0.5 * dy, y2 = -Y + 0.5 * dy;
    const double z1 = -Z - 0.5 * dz, z2 = -Z + 0.5 * dz;
    return pot_corner(a, y2, z2) - pot_corner(a, y1, z2) - pot_corner(a, y2, z1) + pot_corner(a, y1, z1);
}

// S_c at offset (X, Y, Z) of a dx x dy x dz cell
__device__ double pot_kernel(int c, double X, double Y, double Z, double dx, double dy, double dz) {
    const double k = 1.0 / (4.0 * kPiP);
    if (c == 0) return k * (pot_rect(X - 0.5 * dx, Y, Z, dy, dz) - pot_rect(X + 0.5 * dx, Y, Z, dy, dz));
    if (c == 1) return k * (pot_rect(Y - 0.5 * dy, X, Z, dx, dz) - pot_rect(Y + 0.5 * dy, X, Z, dx, dz));
    return k * (pot_rect(Z - 0.5 * dz, X, Y, dx, dy) - pot_rect(Z + 0.5 * dz, X, Y, dx, dy));
}

// offset of padded position p along an axis of n cells and padded length P, or a
// value outside [-n, n] for the positions no offset reaches
__device__ __forceinline__ int pot_offset(int p, int n, int P) {
    if (p <= n) return p;
    if (p >= P - n) return p - P;
    return 1 << 30;
}

// S_c on padded row (y, z) of component c: one CTA per (row, c); complex FFT of
// length Px in shared memory, bins 0..Px/2 to out[c][z][y][kx] (FP64).
__global__ void k_pot_sx(PotGeom g, V2<double>* out, const V2<double>* __restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    V2<double>* a = reinterpret_cast<V2<double>*>(smraw);
    V2<double>* b = a + padded_len(g.Px);
    const int row = blockIdx.x, c = blockIdx.y;
    const int y = row % g.Py, z = row / g.Py;
    const int oy = pot_offset(y, g.ny, g.Py), oz = pot_offset(z, g.nz, g.Pz);
    const bool live = oy != (1 << 30) && oz != (1 << 30);
    for (int x = threadIdx.x; x < g.Px; x += blockDim.x) {
        const int ox = pot_offset(x, g.nx, g.Px);
        double v = 0.0;
        if (live && ox != (1 << 30))
            v = pot_kernel(c, ox * g.dx, oy * g.dy, oz * g.dz, g.dx, g.dy, g.dz);
        a[ix<true>(x, 1)] = mk<double>(v, 0.0);
    }
    __syncthreads();
    const V2<double>* X = stockham_fft<double, false, 3>(a, b, g.lPx, 1, padded_len(g.Px), tw);
    V2<double>* o = out + (((long long)c * g.Pz + z) * g.Py + y) * g.Kx;
    for (int k = threadIdx.x; k < g.Kx; k += blockDim.x) o[k] = X[ix<true>(k, 1)];
}

// M = Ms m on mesh row (y, z) of component c, zero-padded to Px, FFT along x,
// bins 0..Px/2 to out[c][z][y][kx].
template <typename T>
__global__ void k_pot_mx(PotGeom g, const T* __restrict__ m, const T* __restrict__ Ms, T Msu, V2<T>* out,
                         const V2<T>* __restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    V2<T>* a = reinterpret_cast<V2<T>*>(smraw);
    V2<T>* b = a + padded_len(g.Px);
    const int row = blockIdx.x, c = blockIdx.y;
    const int y = row % g.ny, z = row / g.ny;
    const long long N = (long long)g.nx * g.ny * g.nz;
    const long long c0 = ((long long)z * g.ny + y) * g.nx;
    for (int x = threadIdx.x; x < g.Px; x += blockDim.x) {
        T v = (T)0;
        if (x < g.nx) v = (Ms ? Ms[c0 + x] : Msu) * m[c * N + c0 + x];
        a[ix<true>(x, 1)] = mk<T>(v, (T)0);
    }
    __syncthreads();
    const V2<T>* X = stockham_fft<T, false, (sizeof(T) == 4 ? 4 : 3)>(a, b, g.lPx, 1, padded_len(g.Px), tw);
    V2<T>* o = out + (((long long)c * g.Pz + z) * g.Py + y) * g.Kx;
    for (int k = threadIdx.x; k < g.Kx; k += blockDim.x) o[k] = X[ix<true>(k, 1)];
}

// FFT along y (axis 1) or z (axis 2) of buf[nc][Pz][Py][Kx]: one CTA per tile of
// tk consecutive kx columns of one line family.  The first n_in entries of each
// column are read (the rest taken as zero); planes (or rows) beyond `lines` of
// the other transverse axis are not touched.
template <typename T, bool INV>
__global__ void k_pot_col(PotGeom g, V2<T>* buf, int axis, int n_in, int lines, int tk,
                          const V2<T>* __restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int L = axis == 1 ? g.Py : g.Pz, lL = axis == 1 ? g.lPy : g.lPz;
    const int SL = padded_len(L);
    V2<T>* a = reinterpret_cast<V2<T>*>(smraw);
    V2<T>* b = a + tk * SL;
    const int ntile = (g.Kx + tk - 1) / tk;
    const int tile = blockIdx.x % ntile, other = blockIdx.x / ntile;   // other < lines
    const int c = blockIdx.y;
    const int kx0 = tile * tk, nkx = min(tk, g.Kx - kx0);
    long long base, stride;
    if (axis == 1) {   // line (c, z = other, kx): element y at ((c Pz + z) Py + y) Kx + kx
        base = ((long long)c * g.Pz + other) * g.Py * g.Kx + kx0;
        stride = g.Kx;
    } else {           // line (c, y = other, kx): element z at ((c Pz + z) Py + y) Kx + kx
        base = ((long long)c * g.Pz * g.Py + other) * g.Kx + kx0;
        stride = (long long)g.Py * g.Kx;
    }
    for (int i = threadIdx.x; i < L * tk; i += blockDim.x) {
        const int e = i / tk, j = i - e * tk;
        V2<T> v = mk<T>((T)0, (T)0);
        if (e < n_in && j < nkx) v = buf[base + e * stride + j];
        a[j * SL + ix<true>(e, 1)] = v;
    }
    __syncthreads();
    const V2<T>* X = stockham_fft<T, INV, (sizeof(T) == 4 ? 4 : 3)>(a, b, lL, tk, SL, tw);
    for (int i = threadIdx.x; i < L * tk; i += blockDim.x) {
        const int e = i / tk, j = i - e * tk;
        if (j < nkx) buf[base + e * stride + j] = X[j * SL + ix<true>(e, 1)];
    }
}

// u^ = sum_c S^_c M^_c per bin (every bin of the padded half spectrum)
template <typename T>
__global__ void k_pot_dot(long long nbin, const V2<T>* __restrict__ S, const V2<T>* __restrict__ M, V2<T>* U) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nbin;
         i += (long long)gridDim.x * blockDim.x) {
        V2<T> acc = mk<T>((T)0, (T)0);
#pragma unroll
        for (int c = 0; c < 3; ++c) acc = acc + cmul(S[c * nbin + i], M[c * nbin + i]);
        U[i] = acc;
    }
}

// inverse along x of output row (yo, zo), yo = -1..ny, zo = -1..nz: the row's bins
// 0..Px/2 completed by Hermitian symmetry, inverse FFT, positions -1..nx kept in
// u[zo + 1][yo + 1][xo + 1]
template <typename T>
__global__ void k_pot_xinv(PotGeom g, const V2<T>* __restrict__ U, T* u, const V2<T>* __restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    V2<T>* a = reinterpret_cast<V2<T>*>(smraw);
    V2<T>* b = a + padded_len(g.Px);
    const int ey = g.ny + 2;
    const int yo = (int)(blockIdx.x % ey) - 1, zo = (int)(blockIdx.x / ey) - 1;
    const int y = (yo + g.Py) % g.Py, z = (zo + g.Pz) % g.Pz;
    const V2<T>* row = U + ((long long)z * g.Py + y) * g.Kx;
    for (int x = threadIdx.x; x < g.Px; x += blockDim.x) {
        V2<T> v;
        // after the inverse along z and y the row is the x spectrum of a real
        // sequence: X(Px - kx) = conj X(kx)
        v = x < g.Kx ? row[x] : cconj(row[g.Px - x]);
        a[ix<true>(x, 1)] = v;
    }
    __syncthreads();
    const V2<T>* X = stockham_fft<T, true, (sizeof(T) == 4 ? 4 : 3)>(a, b, g.lPx, 1, padded_len(g.Px), tw);
    const int ex = g.nx + 2;
    T* o = u + ((long long)(zo + 1) * ey + (yo + 1)) * ex;
    for (int xo = threadIdx.x; xo < ex; xo += blockDim.x) {
        const int x = (xo - 1 + g.Px) % g.Px;
        o[xo] = X[ix<true>(x, 1)].x;
    }
}

// H_d = -grad u by central differences at every mesh cell
template <typename T>
__global__ void k_pot_grad(PotGeom g, const T* __restrict__ u, T* H) {
    const long long N = (long long)g.nx * g.ny * g.nz;
    const int ex = g.nx + 2, ey = g.ny + 2;
    const T hx = (T)(0.5 / g.dx), hy = (T)(0.5 / g.dy), hz = (T)(0.5 / g.dz);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.nx), y = (int)((i / g.nx) % g.ny), z = (int)(i / ((long long)g.nx * g.ny));
        const long long o = ((long long)(z + 1) * ey + (y + 1)) * ex + (x + 1);
        H[i] = -(u[o + 1] - u[o - 1]) * hx;
        H[N + i] = -(u[o + ex] - u[o - ex]) * hy;
        H[2 * N + i] = -(u[o + (long long)ex * ey] - u[o - (long long)ex * ey]) * hz;
    }
}

// S^ (FP64, unscaled) -> the stored precision, times 1 / (Px Py Pz)
template <typename T>
__global__ void k_pot_store(long long n, const V2<double>* __restrict__ src, V2<T>* dst, double scale) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = mk<T>((T)(src[i].x * scale), (T)(src[i].y * scale));
}

template <typename T>
size_t smem_row(const PotGeom& g) { return 2 * (size_t)padded_len(g.Px) * sizeof(V2<T>); }

// kx columns per column-pass CTA: a tile of at most 48 KB per buffer
template <typename T>
int col_tile(int L) {
    const int cap = (int)(48 * 1024 / (padded_len(L) * sizeof(V2<T>)));
    int tk = 16;
    while (tk > 1 && tk > cap) tk >>= 1;
    return tk;
}

template <typename T>
cudaError_t run_cols(cudaStream_t s, const PotGeom& g, V2<T>* buf, int ncomp, int axis, bool inv, int n_in,
                     int lines, const V2<T>* tw) {
    const int L = axis == 1 ? g.Py : g.Pz;
    if (L <= 1) return cudaSuccess;
    const int tk = col_tile<T>(L);
    const size_t sm = 2 * (size_t)tk * padded_len(L) * sizeof(V2<T>);
    dim3 grid((unsigned)(((g.Kx + tk - 1) / tk) * lines), (unsigned)ncomp);
    if (inv) {
        cudaFuncSetAttribute(k_pot_col<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_pot_col<T, true><<<grid, 256, sm, s>>>(g, buf, axis, n_in, lines, tk, tw);
    } else {
        cudaFuncSetAttribute(k_pot_col<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_pot_col<T, false><<<grid, 256, sm, s>>>(g, buf, axis, n_in, lines, tk, tw);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t pot_field_t(cudaStream_t s, const PotGeom& g, const PotBuffers& B, const void* m, const void* Ms,
                        double Msu, void* H, const void* tw, long long* launches) {
    const V2<T>* twt = reinterpret_cast<const V2<T>*>(tw);
    V2<T>* Mh = reinterpret_cast<V2<T>*>(B.Mhat);
    V2<T>* U = reinterpret_cast<V2<T>*>(B.U);
    const size_t sr = smem_row<T>(g);
    cudaFuncSetAttribute(k_pot_mx<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sr);
    cudaFuncSetAttribute(k_pot_xinv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sr);
    k_pot_mx<T><<<dim3((unsigned)(g.ny * g.nz), 3), 256, sr, s>>>(g, reinterpret_cast<const T*>(m),
                                                                   reinterpret_cast<const T*>(Ms), (T)Msu, Mh, twt);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // y forward on the nz data planes (ny rows in), z forward on every padded row (nz planes in)
    if ((e = run_cols<T>(s, g, Mh, 3, 1, false, g.ny, g.nz, twt)) != cudaSuccess) return e;
    if ((e = run_cols<T>(s, g, Mh, 3, 2, false, g.nz, g.Py, twt)) != cudaSuccess) return e;
    const long long nbin = (long long)g.Pz * g.Py * g.Kx;
    k_pot_dot<T><<<(unsigned)std::min<long long>((nbin + 255) / 256, 4096), 256, 0, s>>>(
        nbin, reinterpret_cast<const V2<T>*>(B.Shat), Mh, U);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the one inverse transform: z, y (every line), then x for the (ny + 2)(nz + 2) rows kept
    if ((e = run_cols<T>(s, g, U, 1, 2, true, g.Pz, g.Py, twt)) != cudaSuccess) return e;
    if ((e = run_cols<T>(s, g, U, 1, 1, true, g.Py, g.Pz, twt)) != cudaSuccess) return e;
    k_pot_xinv<T><<<(unsigned)((g.ny + 2) * (g.nz + 2)), 256, sr, s>>>(g, U, reinterpret_cast<T*>(B.u), twt);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const long long N = (long long)g.nx * g.ny * g.nz;
    k_pot_grad<T><<<(unsigned)std::min<long long>((N + 255) / 256, 4096), 256, 0, s>>>(
        g, reinterpret_cast<const T*>(B.u), reinterpret_cast<T*>(H));
    if (launches) *launches += 5 + (g.Py > 1 ? 2 : 0) + (g.Pz > 1 ? 2 : 0);
    return cudaGetLastError();
}

}  // namespace

PotGeom pot_geometry(int nx, int ny, int nz, double dx, double dy, double dz) {
    PotGeom g;
    g.nx = nx; g.ny = ny; g.nz = nz;
    g.dx = dx; g.dy = dy; g.dz = dz;
    auto pad = [](int n) { int p = 1; while (p < 2 * n + 1) p <<= 1; return p; };
    auto lg = [](int p) { int l = 0; while ((1 << l) < p) ++l; return l; };
    g.Px = pad(nx); g.Py = pad(ny); g.Pz = pad(nz);
    g.lPx = lg(g.Px); g.lPy = lg(g.Py); g.lPz = lg(g.Pz);
    g.Kx = g.Px / 2 + 1;
    return g;
}

long long pot_bins(const PotGeom& g) { return (long long)g.Pz * g.Py * g.Kx; }
long long pot_ext_cells(const PotGeom& g) { return (long long)(g.nx + 2) * (g.ny + 2) * (g.nz + 2); }

cudaError_t pot_precompute(cudaStream_t s, const PotGeom& g, void* Shat, bool f32, void* scratch64, const void* twd,
                           long long* launches) {
    V2<double>* S64 = reinterpret_cast<V2<double>*>(scratch64);
    const V2<double>* tw = reinterpret_cast<const V2<double>*>(twd);
    const size_t sr = smem_row<double>(g);
    cudaFuncSetAttribute(k_pot_sx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sr);
    k_pot_sx<<<dim3((unsigned)(g.Py * g.Pz), 3), 256, sr, s>>>(g, S64, tw);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = run_cols<double>(s, g, S64, 3, 1, false, g.Py, g.Pz, tw)) != cudaSuccess) return e;
    if ((e = run_cols<double>(s, g, S64, 3, 2, false, g.Pz, g.Py, tw)) != cudaSuccess) return e;
    const long long n = 3 * pot_bins(g);
    const double scale = 1.0 / ((double)g.Px * g.Py * g.Pz);
    if (f32)
        k_pot_store<float><<<(unsigned)std::min<long long>((n + 255) / 256, 4096), 256, 0, s>>>(
            n, S64, reinterpret_cast<V2<float>*>(Shat), scale);
    else
        k_pot_store<double><<<(unsigned)std::min<long long>((n + 255) / 256, 4096), 256, 0, s>>>(
            n, S64, reinterpret_cast<V2<double>*>(Shat), scale);
    if (launches) *launches += 2 + (g.Py > 1 ? 1 : 0) + (g.Pz > 1 ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t pot_field(cudaStream_t s, const PotGeom& g, const PotBuffers& B, bool f32, const void* m,
                      const void* Ms, double Msu, void* H, const void* tw, long long* launches) {
    return f32 ? pot_field_t<float>(s, g, B, m, Ms, Msu, H, tw, launches)
               : pot_field_t<double>(s, g, B, m, Ms, Msu, H, tw, launches);
}

}  // namespace mm
