// FP64 precompute of the demagnetising tensor spectrum.
//
// The demag field of a cell mesh is the discrete convolution
// H_d,i = -sum_j N_{i-j} M_j (Sec. "Magnetostatic energy", Eq. 8) with N the
// cell-averaged Newell tensor (Eq. 7; Newell, Williams & Dunlop 1993):
//   * |R| <= 3 max(dx,dy,dz): Newell's closed form -- N_xx is the 27-point
//     second difference (weights 2 at the centre, -1 at +-d, per axis) of
//     f(x,y,z), N_xy the same difference of g(x,y,z), divided by 4 pi dx dy dz;
//     the other components by relabelling axes;
//   * farther out the closed form cancels catastrophically (relative error
//     ~ eps (r/d)^6), so N is evaluated as the average of the point-dipole
//     kernel (r^2 I - 3 r r^T)/(4 pi r^5) times V over the separation t of two
//     points drawn uniformly from the cell: t has density
//     prod_a (1 - |t_a|/d_a)/d_a, integrated per half-tent with q-point
//     Gauss-Legendre (q from 8 down to 3 with distance).
// Both stages run in double precision.  The octant i,j,k >= 0 is evaluated;
// the padded circular arrangement follows from the parities.  Its 3-D FFT
// (FP64) is real; -Re/(Px Py Pz) is stored for the symmetric bins.
#include <math.h>
#include <stdio.h>

#include "engine.cuh"
#include "mm_kernels.cuh"

namespace mm {

__constant__ double c_glu[11][10];   // nodes on [0, 1] of the q-point rule (q = 3..10)
__constant__ double c_glw[11][10];   // tent weights (w/2)(1-u)

// ---- closed form -------------------------------------------------------
__device__ double newell_f(double x, double y, double z) {
    x = fabs(x); y = fabs(y); z = fabs(z);
    const double x2 = x * x, y2 = y * y, z2 = z * z;
    const double R = sqrt(x2 + y2 + z2);
    if (R == 0.0) return 0.0;
    double out = (2.0 * x2 - y2 - z2) * R / 6.0;
    const double rxz = sqrt(x2 + z2), rxy = sqrt(x2 + y2);
    if (rxz > 0.0) out += 0.5 * y * (z2 - x2) * asinh(y / rxz);
    if (rxy > 0.0) out += 0.5 * z * (y2 - x2) * asinh(z / rxy);
    if (x > 0.0) out -= x * y * z * atan(y * z / (x * R));
    return out;
}

__device__ double newell_g(double x, double y, double z) {
    const double sgn = ((x < 0.0) != (y < 0.0)) ? -1.0 : 1.0;
    x = fabs(x); y = fabs(y); z = fabs(z);
    const double x2 = x * x, y2 = y * y, z2 = z * z;
    const double R = sqrt(x2 + y2 + z2);
    if (R == 0.0) return 0.0;
    double out = -x * y * R / 3.0;
    const double rxy = sqrt(x2 + y2), ryz = sqrt(y2 + z2), rxz = sqrt(x2 + z2);
    if (rxy > 0.0) out += x * y * z * asinh(z / rxy);
    if (ryz > 0.0) out += y / 6.0 * (3.0 * z2 - y2) * asinh(x / ryz);
    if (rxz > 0.0) out += x / 6.0 * (3.0 * z2 - x2) * asinh(y / rxz);
    if (z > 0.0) out -= z * z2 / 6.0 * atan(x * y / (z * R));
    if (y > 0.0) out -= z * y2 / 2.0 * atan(x * z / (y * R));
    if (x > 0.0) out -= z * x2 / 2.0 * atan(y * z / (x * R));
    return sgn * out;
}

template <int WHICH>
__device__ double second_diff(double X, double Y, double Z, double dx, double dy, double dz) {
    double acc = 0.0;
    for (int a = -1; a <= 1; ++a) {
        const double wa = a == 0 ? 2.0 : -1.0;
        for (int b = -1; b <= 1; ++b) {
            const double wb = b == 0 ? 2.0 : -1.0;
            for (int c = -1; c <= 1; ++c) {
                const double wc = c == 0 ? 2.0 : -1.0;
                const double x = X + a * dx, y = Y + b * dy, z = Z + c * dz;
                acc += wa * wb * wc * (WHICH == 0 ? newell_f(x, y, z) : newell_g(x, y, z));
            }
        }
    }
    return acc / (4.0 * 3.14159265358979323846 * dx * dy * dz);
}

__device__ void tensor_closed(double X, double Y, double Z, double dx, double dy, double dz, double* t) {
    t[0] = second_diff<0>(X, Y, Z, dx, dy, dz);
    t[1] = second_diff<0>(Y, X, Z, dy, dx, dz);
    t[2] = second_diff<0>(Z, Y, X, dz, dy, dx);
    t[3] = second_diff<1>(X, Y, Z, dx, dy, dz);
    t[4] = second_diff<1>(X, Z, Y, dx, dz, dy);
    t[5] = second_diff<1>(Y, Z, X, dy, dz, dx);
}

// ---- tent-averaged dipole kernel ---------------------------------------
__device__ void tensor_dipole_avg(double X, double Y, double Z, double dx, double dy, double dz, int q,
                                  double* t) {
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int a = 0; a < 2 * q; ++a) {
        const double tx = (a < q ? 1.0 : -1.0) * dx * c_glu[q][a % q];
        const double wx = c_glw[q][a % q];
        const double rx = X + tx;
        for (int b = 0; b < 2 * q; ++b) {
            const double ty = (b < q ? 1.0 : -1.0) * dy * c_glu[q][b % q];
            const double wxy = wx * c_glw[q][b % q];
            const double ry = Y + ty;
            for (int c = 0; c < 2 * q; ++c) {
                const double tz = (c < q ? 1.0 : -1.0) * dz * c_glu[q][c % q];
                const double rz = Z + tz;
                const double r2 = rx * rx + ry * ry + rz * rz;
                const double w = wxy * c_glw[q][c % q] / (r2 * r2 * sqrt(r2));
                acc[0] += w * (r2 - 3.0 * rx * rx);
                acc[1] += w * (r2 - 3.0 * ry * ry);
                acc[2] += w * (r2 - 3.0 * rz * rz);
                acc[3] -= w * 3.0 * rx * ry;
                acc[4] -= w * 3.0 * rx * rz;
                acc[5] -= w * 3.0 * ry * rz;
            }
        }
    }
    const double s = dx * dy * dz / (4.0 * 3.14159265358979323846);
    for (int i = 0; i < 6; ++i) t[i] = acc[i] * s;
}

__device__ int far_nodes(double r_over_d) {
    if (r_over_d <= 4.0) return 8;
    if (r_over_d <= 6.0) return 7;
    if (r_over_d <= 12.0) return 6;
    if (r_over_d <= 32.0) return 5;
    if (r_over_d <= 128.0) return 4;
    return 3;
}

// oct[c][k][j][i] for 0 <= i < nx, 0 <= j < ny, 0 <= k < nz
__global__ void k_newell_octant(int nx, int ny, int nz, double dx, double dy, double dz, double* oct) {
    const long long n = (long long)nx * ny * nz;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n;
         id += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(id % nx);
        const int j = (int)((id / nx) % ny);
        const int k = (int)(id / ((long long)nx * ny));
        const double X = i * dx, Y = j * dy, Z = k * dz;
        const double dmax = fmax(dx, fmax(dy, dz));
        const double r = sqrt(X * X + Y * Y + Z * Z) / dmax;
        double t[6];
        if (r <= 3.0) tensor_closed(X, Y, Z, dx, dy, dz, t);
        else tensor_dipole_avg(X, Y, Z, dx, dy, dz, far_nodes(r), t);
        // off-diagonal components are odd in their two axes: exactly zero on those planes
        if (i == 0 || j == 0) t[3] = 0.0;
        if (i == 0 || k == 0) t[4] = 0.0;
        if (j == 0 || k == 0) t[5] = 0.0;
        for (int c = 0; c < 6; ++c) oct[c * n + id] = t[c];
    }
}

// parity of component c under i -> -i (bit 0), j -> -j (bit 1), k -> -k (bit 2): 1 = odd
__device__ __forceinline__ int odd_mask(int c) {
    switch (c) {
        case 3: return 1 | 2;   // xy
        case 4: return 1 | 4;   // xz
        case 5: return 2 | 4;   // yz
        default: return 0;
    }
}

// circular padded placement of component c into buf[Pz][Py][Px] (complex, imaginary 0)
__global__ void k_newell_place(const double* __restrict__ oct, int c, int nx, int ny, int nz, int Px, int Py,
                               int Pz, double2* buf) {
    const long long n = (long long)nx * ny * nz;
    const long long tot = (long long)Px * Py * Pz;
    const int om = odd_mask(c);
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < tot;
         id += (long long)gridDim.x * blockDim.x) {
        const int X = (int)(id % Px);
        const int Y = (int)((id / Px) % Py);
        const int Z = (int)(id / ((long long)Px * Py));
        int i, j, k;
        double v = 0.0;
        bool ok = true;
        double sign = 1.0;
        if (X < nx) i = X; else if (X > Px - nx) { i = Px - X; if (om & 1) sign = -sign; } else ok = false;
        if (Y < ny) j = Y; else if (Y > Py - ny) { j = Py - Y; if (om & 2) sign = -sign; } else ok = false;
        if (Z < nz) k = Z; else if (Z > Pz - nz) { k = Pz - Z; if (om & 4) sign = -sign; } else ok = false;
        if (ok) v = sign * oct[c * n + ((long long)k * ny + j) * nx + i];
        buf[id] = make_double2(v, 0.0);
    }
}

// in-place forward FFT of every line of buf[Pz][Py][Px] along `axis`
__global__ void k_fft_axis_f64(double2* buf, int Px, int Py, int Pz, int axis, int lL, int TL,
                               const V2<double>* __restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    V2<double>* sm = reinterpret_cast<V2<double>*>(smraw);
    const int L = 1 << lL;
    V2<double>* g = reinterpret_cast<V2<double>*>(buf);
    if (axis == 0) {
        const long long line0 = (long long)blockIdx.x * TL;
        for (int id = threadIdx.x; id < TL * L; id += blockDim.x) {
            const int l = id / L, x = id - l * L;
            sm[l * L + bitrev(x, lL)] = g[(line0 + l) * Px + x];
        }
        __syncthreads();
        fft_dit<double, false>(sm, lL, TL, L, 1, tw);
        for (int id = threadIdx.x; id < TL * L; id += blockDim.x) {
            const int l = id / L, x = id - l * L;
            g[(line0 + l) * Px + x] = sm[l * L + x];
        }
        return;
    }
    // columns: TL adjacent x at fixed (z) for axis 1 or fixed (y) for axis 2
    const int ncolblk = Px / TL;
    const int cb = blockIdx.x % ncolblk;
    const int outer = blockIdx.x / ncolblk;
    const int x0 = cb * TL;
    long long base, estr;
    if (axis == 1) { base = (long long)outer * Py * Px + x0; estr = Px; }
    else { base = (long long)outer * Px + x0; estr = (long long)Px * Py; }
    for (int id = threadIdx.x; id < TL * L; id += blockDim.x) {
        const int col = id % TL, e = id / TL;
        sm[bitrev(e, lL) * TL + col] = g[base + e * estr + col];
    }
    __syncthreads();
    fft_dit<double, false>(sm, lL, TL, 1, TL, tw);
    for (int id = threadIdx.x; id < TL * L; id += blockDim.x) {
        const int col = id % TL, e = id / TL;
        g[base + e * estr + col] = sm[e * TL + col];
    }
}

// Stored tensor values of component c from the transformed buffer:
//   3-D (Ty = 0 or imag_xz = 0 and nk = Pz/2+1): -Re(buf[kz][ky][kx]) * scale for the
//   kz <= Pz/2 bins (the spectrum of an even/odd real tensor is real);
//   films of the cluster pass (nk = nz planes, x and y transformed only):
//   -Re * scale for xx, yy, zz, xy (even in x and y, or odd in both: real) and
//   -Im * scale for xz, yz when imag_xz (odd in exactly one of x, y: imaginary),
//   one value per dz = kz < nz.
// Layout: standard [c][kz][ky][kx]; blocked (Ty > 0) [kx / Ty][ky][kx % Ty][6 kz + c].
// maxim / maxre track the largest discarded and kept parts.
template <typename T>
__global__ void k_newell_extract(const double2* __restrict__ buf, int c, int Px, int Py, int Kx, int Pyh,
                                 int nk, double scale, T* out, int Ty, int qp, int imag_xz,
                                 unsigned long long* maxim, unsigned long long* maxre) {
    const long long tot = (long long)Kx * Pyh * nk;
    const bool im = imag_xz && (c == 4 || c == 5);
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < tot;
         id += (long long)gridDim.x * blockDim.x) {
        const int kx = (int)(id % Kx);
        const int ky = (int)((id / Kx) % Pyh);
        const int kz = (int)(id / ((long long)Kx * Pyh));
        const double2 v = buf[((long long)kz * Py + ky) * Px + kx];
        const double keep = im ? v.y : v.x, drop = im ? v.x : v.y;
        const long long o = Ty > 0 ? (((long long)(kx / Ty) * Pyh + ky) * Ty + kx % Ty) * qp + 6 * kz + c
                                   : (long long)c * tot + id;
        out[o] = T(-keep * scale);
        atomicMax(maxim, (unsigned long long)__double_as_longlong(fabs(drop)));
        atomicMax(maxre, (unsigned long long)__double_as_longlong(fabs(keep)));
    }
}
template __global__ void k_newell_extract<float>(const double2*, int, int, int, int, int, int, double, float*,
                                                  int, int, int, unsigned long long*, unsigned long long*);
template __global__ void k_newell_extract<double>(const double2*, int, int, int, int, int, int, double, double*,
                                                   int, int, int, unsigned long long*, unsigned long long*);
template __global__ void k_newell_extract<dd>(const double2*, int, int, int, int, int, int, double, dd*,
                                               int, int, int, unsigned long long*, unsigned long long*);

// twiddle tables: exp(-2 pi i k / LMAX) for k < LMAX, then the stage tables
// W_M^(k r) (layout: stw_base in mm_kernels.cuh), all from FP64 sincospi of the
// exact fraction 2 (k r mod M) / M
__global__ void k_twiddles(V2<double>* twd, V2<float>* twf, V2<dd>* twdd) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < MM_TW_ENTRIES; i += gridDim.x * blockDim.x) {
        long long num;
        int lM;
        if (i < MM_LMAX) {
            num = i;
            lM = MM_LOG2_LMAX;
        } else {
            int rem = i - MM_LMAX, LR = 1;
            while (LR < 4 && rem >= stw_off(LR + 1)) ++LR;
            rem -= stw_off(LR);
            const int R1 = (1 << LR) - 1;
            lM = LR;
            while (rem >= R1 * (1 << (lM - LR))) { rem -= R1 * (1 << (lM - LR)); ++lM; }
            const int ns = 1 << (lM - LR);
            const int r = rem / ns + 1, k = rem - (r - 1) * ns;
            num = ((long long)k * r) & ((1LL << lM) - 1);
        }
        double s, c;
        sincospi(2.0 * (double)num / (double)(1LL << lM), &s, &c);
        twd[i].x = c; twd[i].y = -s;
        twf[i].x = (float)c; twf[i].y = (float)-s;
        if (twdd) { twdd[i].x = dd(c); twdd[i].y = dd(-s); }
    }
}

// ---- host side ----------------------------------------------------------
// Gauss-Legendre nodes by Newton iteration on P_q; mapped to the half-tent
// integral  int_0^1 (1-u) phi(u) du  ~  sum_k W_k phi(u_k).
void upload_gauss_legendre() {
    double U[11][10] = {}, W[11][10] = {};
    for (int q = 3; q <= 10; ++q) {
        for (int i = 0; i < q; ++i) {
            double x = cos(3.14159265358979323846 * (i + 0.75) / (q + 0.5));
            for (int it = 0; it < 100; ++it) {
                double p0 = 1.0, p1 = x;
                for (int k = 2; k <= q; ++k) {
                    const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                    p0 = p1; p1 = p2;
                }
                const double dp = q * (x * p1 - p0) / (x * x - 1.0);
                const double dx = p1 / dp;
                x -= dx;
                if (fabs(dx) < 1e-16) break;
            }
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= q; ++k) {
                const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            const double dp = q * (x * p1 - p0) / (x * x - 1.0);
            const double w = 2.0 / ((1.0 - x * x) * dp * dp);
            const double u = 0.5 * (1.0 + x);
            U[q][i] = u;
            W[q][i] = 0.5 * w * (1.0 - u);
        }
    }
    cudaMemcpyToSymbol(c_glu, U, sizeof(U));
    cudaMemcpyToSymbol(c_glw, W, sizeof(W));
}

// ---- launch wrappers ------------------------------------------------------
void launch_twiddles(cudaStream_t s, void* twd, void* twf, void* twdd) {
    k_twiddles<<<32, 256, 0, s>>>(reinterpret_cast<V2<double>*>(twd), reinterpret_cast<V2<float>*>(twf),
                                  reinterpret_cast<V2<dd>*>(twdd));
}

void launch_newell_octant(cudaStream_t s, int nx, int ny, int nz, double dx, double dy, double dz, double* oct) {
    const long long n = (long long)nx * ny * nz;
    const long long blocks = (n + 127) / 128;
    k_newell_octant<<<(int)(blocks < 1048576 ? blocks : 1048576), 128, 0, s>>>(nx, ny, nz, dx, dy, dz, oct);
}

void launch_newell_place(cudaStream_t s, const double* oct, int c, int nx, int ny, int nz, int Px, int Py, int Pz,
                         void* buf) {
    const long long n = (long long)Px * Py * Pz;
    const long long blocks = (n + 255) / 256;
    k_newell_place<<<(int)(blocks < 1048576 ? blocks : 1048576), 256, 0, s>>>(oct, c, nx, ny, nz, Px, Py, Pz,
                                                                             reinterpret_cast<double2*>(buf));
}

void launch_fft_axis_f64(cudaStream_t s, void* buf, int Px, int Py, int Pz, int axis, const void* twd) {
    const int L = axis == 0 ? Px : (axis == 1 ? Py : Pz);
    if (L <= 1) return;
    int lL = 0;
    while ((1 << lL) < L) ++lL;
    // lines per CTA: keep the tile at >= 4096 elements (64 KB), at least 1
    int TL = L >= 4096 ? 1 : 4096 / L;
    long long blocks;
    if (axis == 0) {
        const long long lines = (long long)Py * Pz;
        if (TL > lines) TL = (int)lines;
        blocks = lines / TL;
    } else {
        if (TL > Px) TL = Px;
        blocks = (long long)(Px / TL) * (axis == 1 ? Pz : Py);
    }
    const size_t smem = (size_t)TL * L * sizeof(double2);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_fft_axis_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        attr = true;
    }
    k_fft_axis_f64<<<(unsigned)blocks, 256, smem, s>>>(reinterpret_cast<double2*>(buf), Px, Py, Pz, axis, lL, TL,
                                                       reinterpret_cast<const V2<double>*>(twd));
}

void launch_newell_extract(cudaStream_t s, const void* buf, int c, int Px, int Py, int Kx, int Pyh, int nk,
                           double scale, void* out, int out_kind, int Ty, int qp, int imag_xz,
                           unsigned long long* maxim, unsigned long long* maxre) {
    const long long n = (long long)Kx * Pyh * nk;
    const long long blocks = (n + 255) / 256;
    const int g = (int)(blocks < 1048576 ? blocks : 1048576);
    if (out_kind == 1)
        k_newell_extract<float><<<g, 256, 0, s>>>(reinterpret_cast<const double2*>(buf), c, Px, Py, Kx, Pyh, nk,
                                                   scale, reinterpret_cast<float*>(out), Ty, qp, imag_xz, maxim,
                                                   maxre);
    else if (out_kind == 2)
        k_newell_extract<dd><<<g, 256, 0, s>>>(reinterpret_cast<const double2*>(buf), c, Px, Py, Kx, Pyh, nk,
                                                scale, reinterpret_cast<dd*>(out), Ty, qp, imag_xz, maxim, maxre);
    else
        k_newell_extract<double><<<g, 256, 0, s>>>(reinterpret_cast<const double2*>(buf), c, Px, Py, Kx, Pyh, nk,
                                                    scale, reinterpret_cast<double*>(out), Ty, qp, imag_xz, maxim,
                                                    maxre);
}

}  // namespace mm
