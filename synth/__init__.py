"""Seeded synthetic inputs shared by the CUDA path and the FP64 oracle.

This module only builds inputs: meshes, material tables and initial
magnetisation states drawn from a counter-based SplitMix64 stream
(Steele, Lea & Flood 2014).  It holds none of the solver's arithmetic
(no fields, no torques, no integrator).  Both sides of every parity test
receive the same arrays from here.

Array convention: a magnetisation state is a float64 array of shape
(3, nz, ny, nx) -- structure of arrays, x fastest -- with unit vectors in
every cell.  Lengths are metres, fields A/m, energies J.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np

MU0 = 4e-7 * math.pi                      # vacuum permeability (exact SI definition used here)
MT = 1e-3 / MU0                           # 1 mT of mu0*H expressed in A/m

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """The outputs start..start+n-1 of SplitMix64 seeded with `seed`.

    Output k is mix(seed + (k+1)*0x9E3779B97F4A7C15), the published
    finaliser of Steele, Lea & Flood (2014), so any slice of the stream can
    be produced without generating the prefix.
    """
    with np.errstate(over="ignore"):
        k = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, start: int = 0) -> np.ndarray:
    """n doubles in [0, 1): the top 53 bits of each SplitMix64 output."""
    return (splitmix64(seed, n, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def random_unit_vectors(seed: int, n: int) -> np.ndarray:
    """n i.i.d. unit vectors, uniform on the sphere; shape (3, n).

    z = 2u - 1 and phi = 2*pi*v with (u, v) consecutive uniforms.
    """
    uv = uniform(seed, 2 * n).reshape(n, 2)
    z = 2.0 * uv[:, 0] - 1.0
    phi = 2.0 * math.pi * uv[:, 1]
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([s * np.cos(phi), s * np.sin(phi), z])


# --------------------------------------------------------------------------
# meshes and materials
# --------------------------------------------------------------------------

@dataclass
class Mesh:
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


@dataclass
class Material:
    """Per-simulation material constants (SI)."""
    Ms: float
    A: float = 0.0
    D: float = 0.0
    dmi: int = 0                  # 0 none, 1 interfacial (C_nv), 2 bulk (T, O), 3 D_2d
    Ku: float = 0.0
    u: tuple = (0.0, 0.0, 1.0)
    Kc: float = 0.0               # cubic, energy density Kc*(mx^4+my^4+mz^4)
    H: tuple = (0.0, 0.0, 0.0)    # applied field, A/m
    alpha: float = 0.5
    gamma: float = 2.211e5
    precession: int = 1
    demag: int = 1
    # per-cell exchange / DMI constants (nz, ny, nx), None for the uniform A / D
    A_cells: Optional[np.ndarray] = None
    D_cells: Optional[np.ndarray] = None
    # spin-transfer torque (Zhang-Li): drift velocity u (m/s), non-adiabaticity beta
    u_stt: tuple = (0.0, 0.0, 0.0)
    beta: float = 0.0
    # Slonczewski / spin-orbit torque: a_J, b_J (1/s) and polarisation p
    aJ: float = 0.0
    bJ: float = 0.0
    p: tuple = (0.0, 0.0, 1.0)


@dataclass
class Sim:
    mesh: Mesh
    mat: Material
    m0: np.ndarray                          # (3, nz, ny, nx)
    Ms_cells: Optional[np.ndarray] = None   # (nz, ny, nx) or None for uniform Ms


@dataclass
class Workload:
    name: str
    sims: List[Sim]
    precision: str                 # "f64" or "f32"
    rtol: float
    t_end: float = 0.0
    steps: int = 0
    neb: dict = field(default_factory=dict)
    sweep_mT: Optional[np.ndarray] = None
    max_dmdt: float = 0.0          # rad/s


def uniform_state(mesh: Mesh, direction=(0.0, 0.0, 1.0)) -> np.ndarray:
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    m = np.empty((3,) + mesh.shape)
    for c in range(3):
        m[c] = d[c]
    return m


def random_state(seed: int, mesh: Mesh) -> np.ndarray:
    return random_unit_vectors(seed, mesh.ncells).reshape((3,) + mesh.shape)


def skyrmion_disks(seed: int, mesh: Mesh, count: int = 200, rmin: float = 6e-9,
                   rmax: float = 12e-9, gap: float = 2e-9, wall: float = 2e-9,
                   max_tries: int = 100000) -> np.ndarray:
    """Reversed Neel-type disks in a +z background (all layers).

    Centres uniform over the film, radii uniform in [rmin, rmax]; a centre is
    rejected when it lies closer than r1 + r2 + gap to an accepted one.  Each
    cell takes the profile of its nearest disk:
    theta(r) = 2*atan(exp((R - r)/wall)), m = (sin th cos phi, sin th sin phi, cos th),
    phi the azimuth around the disk centre.
    """
    Lx, Ly = mesh.nx * mesh.dx, mesh.ny * mesh.dy
    rnd = uniform(seed, 3 * max_tries).reshape(max_tries, 3)
    cx, cy, rr = [], [], []
    for t in range(max_tries):
        if len(rr) >= count:
            break
        x0, y0 = rnd[t, 0] * Lx, rnd[t, 1] * Ly
        r0 = rmin + (rmax - rmin) * rnd[t, 2]
        ok = True
        for (a, b, r) in zip(cx, cy, rr):
            if (a - x0) ** 2 + (b - y0) ** 2 < (r + r0 + gap) ** 2:
                ok = False
                break
        if ok:
            cx.append(x0); cy.append(y0); rr.append(r0)
    cx, cy, rr = np.array(cx), np.array(cy), np.array(rr)
    xs = (np.arange(mesh.nx) + 0.5) * mesh.dx
    ys = (np.arange(mesh.ny) + 0.5) * mesh.dy
    X, Y = np.meshgrid(xs, ys)                      # (ny, nx)
    best = np.full(X.shape, np.inf)
    theta = np.zeros(X.shape)
    phi = np.zeros(X.shape)
    for a, b, r in zip(cx, cy, rr):
        dxp, dyp = X - a, Y - b
        dist = np.sqrt(dxp * dxp + dyp * dyp)
        near = (dist - r) < best
        best = np.where(near, dist - r, best)
        th = 2.0 * np.arctan(np.exp(np.clip((r - dist) / wall, -700, 700)))
        theta = np.where(near, th, theta)
        phi = np.where(near, np.arctan2(dyp, dxp), phi)
    m2 = np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)])
    m = np.empty((3,) + mesh.shape)
    for z in range(mesh.nz):
        m[:, z] = m2
    return m


def voronoi_domains(seed: int, mesh: Mesh, k: int = 64) -> np.ndarray:
    """Each cell takes the direction of its nearest of k seeded sites.

    Sites are uniform in the box (cell-index units); their directions are
    uniform on the sphere.  Distances are Euclidean in metres.
    """
    u = uniform(seed, 3 * k).reshape(k, 3)
    sites = u * np.array([mesh.nx * mesh.dx, mesh.ny * mesh.dy, mesh.nz * mesh.dz])
    dirs = random_unit_vectors(seed ^ 0x5DEECE66D, k)          # (3, k)
    xs = (np.arange(mesh.nx) + 0.5) * mesh.dx
    ys = (np.arange(mesh.ny) + 0.5) * mesh.dy
    Y, X = np.meshgrid(ys, xs, indexing="ij")                   # (ny, nx)
    m = np.empty((3,) + mesh.shape)
    for z in range(mesh.nz):
        zc = (z + 0.5) * mesh.dz
        best = np.full(X.shape, np.inf)
        idx = np.zeros(X.shape, dtype=np.int64)
        for s in range(k):
            d2 = (X - sites[s, 0]) ** 2 + (Y - sites[s, 1]) ** 2 + (zc - sites[s, 2]) ** 2
            near = d2 < best
            best = np.where(near, d2, best)
            idx = np.where(near, s, idx)
        m[:, z] = dirs[:, idx]
    return m


def tilt(m: np.ndarray, seed: int, angle: float) -> np.ndarray:
    """Add a seeded random perturbation of size ~angle (rad) and renormalise."""
    n = m[0].size
    r = random_unit_vectors(seed, n).reshape(m.shape)
    out = m + angle * r
    return out / np.sqrt((out * out).sum(axis=0))


def geodesic_chain(m_a: np.ndarray, m_b: np.ndarray, n_images: int) -> np.ndarray:
    """Initial NEB path: per-cell great-circle interpolation (slerp).

    Image i of n_images sits at fraction s = i/(n_images-1).  For a cell
    where m_a and m_b are antiparallel the rotation axis is e_x x m_a, or
    e_y x m_a when that vanishes.  Returns shape (n_images, 3, nz, ny, nx).
    """
    a = m_a.reshape(3, -1)
    b = m_b.reshape(3, -1)
    dot = np.clip((a * b).sum(axis=0), -1.0, 1.0)
    ang = np.arccos(dot)
    # rotation axis (unit) k with b = rotation of a about k by ang
    k = np.cross(a.T, b.T).T
    kn = np.sqrt((k * k).sum(axis=0))
    degenerate = kn < 1e-12
    ex = np.zeros_like(a); ex[0] = 1.0
    ey = np.zeros_like(a); ey[1] = 1.0
    kx = np.cross(ex.T, a.T).T
    kxn = np.sqrt((kx * kx).sum(axis=0))
    ky = np.cross(ey.T, a.T).T
    alt = np.where(kxn > 1e-12, kx / np.maximum(kxn, 1e-300), ky / np.maximum(np.sqrt((ky * ky).sum(axis=0)), 1e-300))
    k = np.where(degenerate, alt, k / np.maximum(kn, 1e-300))
    out = np.empty((n_images,) + m_a.shape)
    for i in range(n_images):
        s = i / (n_images - 1)
        th = s * ang
        c, sn = np.cos(th), np.sin(th)
        kxa = np.cross(k.T, a.T).T
        kda = (k * a).sum(axis=0)
        v = a * c + kxa * sn + k * kda * (1.0 - c)          # Rodrigues rotation
        v = v / np.sqrt((v * v).sum(axis=0))
        out[i] = v.reshape(m_a.shape)
    out[0] = m_a
    out[-1] = m_b
    return out


# --------------------------------------------------------------------------
# the five workloads (film relax, thin film, bulk cube, NEB chain, uneven batch)
# --------------------------------------------------------------------------

def film_relax_32(seed: int = 1) -> Workload:
    """32x32x1 Py-like film, exchange + demag + 10 mT along +x, random start, 1 ns."""
    mesh = Mesh(32, 32, 1, 2.5e-9, 2.5e-9, 3e-9)
    mat = Material(Ms=8.6e5, A=1.3e-11, alpha=0.5, gamma=2.211e5, H=(10 * MT, 0.0, 0.0))
    return Workload("film_relax_32x32x1_f64", [Sim(mesh, mat, random_state(seed, mesh))],
                    precision="f64", rtol=1e-6, t_end=1e-9)


def skyrmion_film(seed: int = 2, nx: int = 512, ny: int = 512, nz: int = 4,
                  count: int = 200, precision: str = "f32") -> Workload:
    """Thin film with interfacial DMI and perpendicular anisotropy, reversed disks."""
    mesh = Mesh(nx, ny, nz, 2e-9, 2e-9, 1e-9)
    mat = Material(Ms=5.8e5, A=1.5e-11, D=3e-3, dmi=1, Ku=8e5, u=(0.0, 0.0, 1.0), alpha=0.1)
    m0 = skyrmion_disks(seed, mesh, count=count)
    return Workload(f"skyrmion_film_{nx}x{ny}x{nz}_{precision}", [Sim(mesh, mat, m0)],
                    precision=precision, rtol=1e-6 if precision == "f64" else 1e-5, steps=2000)


def bulk_cube(seed: int = 3, n: int = 256, precision: str = "f32") -> Workload:
    """Iron-like cube, cubic anisotropy K1 = 4.8e4 J/m^3 (Kc = -K1/2), Voronoi start."""
    mesh = Mesh(n, n, n, 3e-9, 3e-9, 3e-9)
    mat = Material(Ms=1.7e6, A=2.1e-11, Kc=-2.4e4, alpha=0.02)
    return Workload(f"bulk_cube_{n}^3_{precision}", [Sim(mesh, mat, voronoi_domains(seed, mesh, 64))],
                    precision=precision, rtol=1e-6 if precision == "f64" else 1e-5, steps=200)


def neb_chain(seed: int = 4, n_images: int = 32, n: int = 128, precision: str = "f32",
              radius: float = 8e-9) -> Workload:
    """Skyrmion-collapse NEB chain: single skyrmion -> uniform +z, geodesic start."""
    mesh = Mesh(n, n, 1, 1e-9, 1e-9, 0.5e-9)
    mat = Material(Ms=5.8e5, A=1.5e-11, D=3e-3, dmi=1, Ku=8e5, u=(0.0, 0.0, 1.0),
                   alpha=0.5, precession=0)
    # one disk at the centre
    xs = (np.arange(n) + 0.5) * mesh.dx - 0.5 * n * mesh.dx
    X, Y = np.meshgrid(xs, xs)
    r = np.sqrt(X * X + Y * Y)
    th = 2.0 * np.arctan(np.exp(np.clip((radius - r) / 2e-9, -700, 700)))
    ph = np.arctan2(Y, X)
    sk = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])[:, None]
    up = uniform_state(mesh, (0, 0, 1))
    chain = geodesic_chain(sk, up, n_images)
    sims = [Sim(mesh, mat, chain[i]) for i in range(n_images)]
    return Workload(f"neb_{n_images}x{n}x{n}x1_{precision}", sims, precision=precision,
                    rtol=1e-5, steps=500, neb={"k_spring": 1e5, "n_images": n_images})


def square_film(n: int, seed: int = 6, precision: str = "f32") -> Workload:
    """N x N x 1 film with demag, exchange and Zeeman only, random start (the
    mesh family of the paper's throughput comparison, Sec. 4 'Performance')."""
    mesh = Mesh(n, n, 1, 2e-9, 2e-9, 2e-9)
    mat = Material(Ms=8e5, A=1.3e-11, alpha=0.1, H=(0.0, 0.0, 10 * MT))
    return Workload(f"square_film_{n}x{n}x1_{precision}", [Sim(mesh, mat, random_state(seed, mesh))],
                    precision=precision, rtol=1e-6 if precision == "f64" else 1e-5)


MESH_CHOICES = [(64, 64, 1), (128, 64, 2), (256, 256, 1), (512, 256, 4)]


def uneven_batch(seed: int = 5, count: int = 64, precision: str = "f32",
                 choices=None) -> Workload:
    """count independent simulations, meshes and materials drawn per simulation."""
    choices = MESH_CHOICES if choices is None else choices
    u = uniform(seed, 8 * count).reshape(count, 8)
    sims = []
    for s in range(count):
        nx, ny, nz = choices[min(int(u[s, 0] * len(choices)), len(choices) - 1)]
        mesh = Mesh(nx, ny, nz, 2e-9, 2e-9, 2e-9)
        mat = Material(Ms=4e5 + u[s, 1] * 8e5, A=0.5e-11 + u[s, 2] * 1.5e-11,
                       D=u[s, 3] * 4e-3, dmi=1, Ku=u[s, 4] * 1e6, u=(0.0, 0.0, 1.0),
                       alpha=0.01 + u[s, 5] * 0.49, precession=0, H=(0.0, 0.0, -100 * MT))
        m0 = tilt(uniform_state(mesh, (0, 0, -1)), seed * 1000 + s, 0.01)
        sims.append(Sim(mesh, mat, m0))
    return Workload(f"uneven_batch_{count}_{precision}", sims, precision=precision, rtol=1e-5,
                    sweep_mT=np.linspace(-100.0, 100.0, 41), max_dmdt=1e7)


def with_precision(w: Workload, precision: str) -> Workload:
    return replace(w, precision=precision)


def with_extended_terms(w: Workload, seed: int = 7) -> Workload:
    """The workload with per-cell exchange and DMI constants (uniform within +-10 % of
    the material's) and a Zhang-Li drift u = (50, 0, 0) m/s, beta = 0.1: inputs that
    run the extended epilogue on the same meshes and states."""
    sims = []
    for i, s in enumerate(w.sims):
        r = uniform(seed + i, 2 * s.mesh.ncells).reshape((2,) + s.mesh.shape)
        mat = replace(s.mat, A_cells=s.mat.A * (0.9 + 0.2 * r[0]), D_cells=s.mat.D * (0.9 + 0.2 * r[1]),
                      u_stt=(50.0, 0.0, 0.0), beta=0.1)
        sims.append(replace(s, mat=mat))
    return replace(w, name=w.name + "_ext", sims=sims)
