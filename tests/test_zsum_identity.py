"""The z part of the demag convolution (Eq. 8) written as a sum over planes.

Films of 2..8 planes transform the Newell tensor along x and y only and form
H(kx, ky, z) = sum_z' Nhat(kx, ky, z - z') M(kx, ky, z') directly.  In that
mixed domain the xx, yy, zz, xy components are real and xz, yz purely
imaginary (odd in exactly one of x, y), offsets dz < 0 follow from the z
parities (xz, yz odd) and ky > Py/2 from the y parities (xy, yz odd).  This
pins those facts against the zero-padded 3-D FFT product they replace, on a
random tensor with the Newell tensor's parities, in numpy (no GPU, no oracle).
"""
import numpy as np
import pytest

ODD = {0: 0, 1: 0, 2: 0, 3: 0b011, 4: 0b101, 5: 0b110}   # xx yy zz xy xz yz: odd in x=1, y=2, z=4
PAIR = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (0, 1): 3, (1, 0): 3, (0, 2): 4, (2, 0): 4, (1, 2): 5, (2, 1): 5}


def _pad(n, min2=False):
    if n <= 1:
        return 2 if min2 else 1
    p = 1
    while p < 2 * n - 1:
        p *= 2
    return p


def _placed(rng, nx, ny, nz, P):
    """Circular zero-padded placement of random offsets |i| < n with the tensor parities."""
    Px, Py, Pz = P
    out = []
    for c in range(6):
        t = rng.standard_normal((nz, ny, nx))
        if ODD[c] & 1:
            t[:, :, 0] = 0
        if ODD[c] & 2:
            t[:, 0, :] = 0
        if ODD[c] & 4:
            t[0, :, :] = 0
        g = np.zeros((Pz, Py, Px))
        for k in range(-(nz - 1), nz):
            for j in range(-(ny - 1), ny):
                for i in range(-(nx - 1), nx):
                    s = 1.0
                    s *= -1.0 if (i < 0 and ODD[c] & 1) else 1.0
                    s *= -1.0 if (j < 0 and ODD[c] & 2) else 1.0
                    s *= -1.0 if (k < 0 and ODD[c] & 4) else 1.0
                    g[k % Pz, j % Py, i % Px] = s * t[abs(k), abs(j), abs(i)]
        out.append(g)
    return out


@pytest.mark.parametrize("n", [(5, 6, 2), (4, 3, 3), (6, 5, 4), (3, 4, 8)])
def test_plane_sum_equals_padded_fft_product(n):
    nx, ny, nz = n
    P = (_pad(nx, True), _pad(ny), _pad(nz))
    Px, Py, Pz = P
    rng = np.random.default_rng(sum(n))
    G = _placed(rng, nx, ny, nz, P)
    M = rng.standard_normal((3, nz, Py, Px)) + 1j * rng.standard_normal((3, nz, Py, Px))
    # zero-padded 3-D product: the spectrum of the tensor is real
    T3 = [-np.real(np.fft.fftn(g)) / (Px * Py * Pz) for g in G]
    Mp = np.zeros((3, Pz, Py, Px), complex)
    Mp[:, :nz] = M
    Mh = np.fft.fft(Mp, axis=1)
    HA = np.zeros_like(Mh)
    for a in range(3):
        for b in range(3):
            HA[a] += T3[PAIR[(a, b)]] * Mh[b]
    HA = (np.fft.ifft(HA, axis=1) * Pz)[:, :nz]
    # x-y transform only: real or imaginary per component, then the plane sum
    T2 = []
    for c in range(6):
        F = np.fft.fft2(G[c])
        keep, drop = (F.imag, F.real) if c in (4, 5) else (F.real, F.imag)
        assert np.abs(drop).max() <= 1e-10 * np.abs(keep).max()
        T2.append(-keep[:nz] / (Px * Py))
    HB = np.zeros((3, nz, Py, Px), complex)
    for z in range(nz):
        for z2 in range(nz):
            dz, so = abs(z - z2), (1.0 if z >= z2 else -1.0)
            xx, yy, zz, xy = T2[0][dz], T2[1][dz], T2[2][dz], T2[3][dz]
            xz, yz = so * T2[4][dz], so * T2[5][dz]
            a, b, c = M[0, z2], M[1, z2], M[2, z2]
            HB[0, z] += xx * a + xy * b + 1j * xz * c
            HB[1, z] += xy * a + yy * b + 1j * yz * c
            HB[2, z] += 1j * xz * a + 1j * yz * b + zz * c
    assert np.abs(HA - HB).max() <= 1e-12 * np.abs(HA).max()
    # ky > Py/2 is the ky fold of the stored half: xy and yz change sign
    for c in range(6):
        F = np.fft.fft2(G[c])
        keep = F.imag if c in (4, 5) else F.real
        sy = -1.0 if c in (3, 5) else 1.0
        for ky in range(Py // 2 + 1, Py):
            assert np.allclose(keep[:, ky, :], sy * keep[:, Py - ky, :], rtol=0, atol=1e-12 * np.abs(keep).max())
