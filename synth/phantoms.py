"""Seeded synthetic phantoms, sources and random vectors.

Conventions shared by every consumer:
  * a grid of Nx x Ny x Nz voxels with side lengths (dx, dy, dz) in metres, the
    box centred at the origin; voxel (ix, iy, iz) has its centre at
    ((ix + 1/2 - Nx/2) dx, (iy + 1/2 - Ny/2) dy, (iz + 1/2 - Nz/2) dz);
  * per-voxel maps are C-ordered float64 arrays of shape (Nz, Ny, Nx);
  * a voxel takes the material found at its centre (the staircase rule of the
    piecewise-constant material model, Section III-A, Eq. 23);
  * air is eps_real = 1, sigma = 0.

Nothing here evaluates the integral-equation method; the complex permittivity
eps_real - i sigma / (omega eps0) is formed by each consumer.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Grid:
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def nv(self):
        return self.nx * self.ny * self.nz

    def centres(self):
        """Voxel-centre coordinates as three (Nz, Ny, Nx) arrays (x, y, z)."""
        x = (np.arange(self.nx) + 0.5 - self.nx / 2.0) * self.dx
        y = (np.arange(self.ny) + 0.5 - self.ny / 2.0) * self.dy
        z = (np.arange(self.nz) + 0.5 - self.nz / 2.0) * self.dz
        zz, yy, xx = np.meshgrid(z, y, x, indexing="ij")
        return xx, yy, zz


# Synthetic four-shell tissue model: (scale of the outer ellipsoid, eps_real, sigma S/m),
# outermost first.  These are synthetic values, not a tissue database.
_SHELLS = ((1.00, 40.0, 0.60), (0.92, 15.0, 0.10), (0.85, 75.0, 2.00), (0.60, 52.0, 0.55))


def _smoothed_noise(shape, seed, sigma_vox=2.0):
    from scipy.ndimage import gaussian_filter

    rng = np.random.Generator(np.random.PCG64(seed))
    n = rng.standard_normal(shape)
    n = gaussian_filter(n, sigma=sigma_vox, mode="reflect")
    n = n - n.mean()
    sd = n.std()
    return n / sd if sd > 0 else n


def _shelled(grid: Grid, ellipsoids, seed, amplitude=0.15):
    """Nested-shell ellipsoid union with multiplicative smoothed noise.

    ellipsoids: iterable of ((cx, cy, cz), (ax, ay, az)) in metres.
    Returns (eps_real, sigma) maps; air outside every ellipsoid.
    """
    xx, yy, zz = grid.centres()
    shell = np.full(grid.shape, -1, dtype=np.int64)
    for (cx, cy, cz), (ax, ay, az) in ellipsoids:
        rho2 = ((xx - cx) / ax) ** 2 + ((yy - cy) / ay) ** 2 + ((zz - cz) / az) ** 2
        for s, (scale, _, _) in enumerate(_SHELLS):
            inside = rho2 <= scale * scale
            shell = np.where(inside & (shell < s), s, shell)
    eps = np.ones(grid.shape)
    sig = np.zeros(grid.shape)
    noise = _smoothed_noise(grid.shape, seed)
    for s, (_, e, c) in enumerate(_SHELLS):
        m = shell == s
        eps[m] = e * (1.0 + amplitude * noise[m])
        sig[m] = c * (1.0 + amplitude * noise[m])
    tissue = shell >= 0
    eps[tissue] = np.clip(eps[tissue], 5.0, 80.0)
    sig[tissue] = np.clip(sig[tissue], 0.05, 2.0)
    return eps, sig


def sphere_phantom(grid: Grid, radius, eps_real, sigma, centre=(0.0, 0.0, 0.0)):
    """Homogeneous sphere, centre-in voxelisation."""
    xx, yy, zz = grid.centres()
    inside = (xx - centre[0]) ** 2 + (yy - centre[1]) ** 2 + (zz - centre[2]) ** 2 <= radius * radius
    eps = np.where(inside, float(eps_real), 1.0)
    sig = np.where(inside, float(sigma), 0.0)
    return eps, sig


def head_phantom(grid: Grid, seed=1234, semi_axes=(0.09, 0.07, 0.11)):
    """Head-size ellipsoid with four nested shells plus smoothed noise, clipped by the box."""
    return _shelled(grid, [((0.0, 0.0, 0.0), semi_axes)], seed)


def body_phantom(grid: Grid, seed=1235):
    """Torso / neck / head stack of ellipsoids with the same shell and noise model."""
    ell = [
        ((0.0, 0.0, -0.25), (0.17, 0.11, 0.30)),
        ((0.0, 0.0, 0.10), (0.06, 0.06, 0.08)),
        ((0.0, 0.0, 0.26), (0.09, 0.07, 0.11)),
    ]
    return _shelled(grid, ell, seed)


def inclusion_phantom(grid: Grid, seed=99, n_incl=8, bg=(5.0, 0.05), incl=(80.0, 2.0)):
    """High-contrast spherical inclusions (radius 4-10 voxels) in a background filling the box."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xx, yy, zz = grid.centres()
    eps = np.full(grid.shape, bg[0])
    sig = np.full(grid.shape, bg[1])
    h = min(grid.dx, grid.dy, grid.dz)
    half = np.array([grid.nx * grid.dx, grid.ny * grid.dy, grid.nz * grid.dz]) / 2.0
    for _ in range(n_incl):
        r = rng.uniform(4.0, 10.0) * h
        c = rng.uniform(-half + r, half - r)
        m = (xx - c[0]) ** 2 + (yy - c[1]) ** 2 + (zz - c[2]) ** 2 <= r * r
        eps[m] = incl[0]
        sig[m] = incl[1]
    return eps, sig


def random_tissue(grid: Grid, seed, air_fraction=0.2):
    """Independent random materials per voxel (eps_real in [1, 80], sigma in [0, 2]) with some air."""
    rng = np.random.Generator(np.random.PCG64(seed))
    eps = rng.uniform(1.0, 80.0, grid.shape)
    sig = rng.uniform(0.0, 2.0, grid.shape)
    air = rng.uniform(0.0, 1.0, grid.shape) < air_fraction
    eps[air] = 1.0
    sig[air] = 0.0
    return eps, sig


def random_permeability(grid: Grid, seed, nonmagnetic_fraction=0.3):
    """Independent random relative permeability per voxel, mu = mu_real - i mu_imag with
    mu_real in [1, 4] and mu_imag in [0, 1], and mu = 1 in some voxels (synthetic
    magnetodielectric material for the full JM-VIE; tissue itself is non-magnetic)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mr = rng.uniform(1.0, 4.0, grid.shape)
    mi = rng.uniform(0.0, 1.0, grid.shape)
    plain = rng.uniform(0.0, 1.0, grid.shape) < nonmagnetic_fraction
    mr[plain] = 1.0
    mi[plain] = 0.0
    return mr, mi


def ring_dipoles(n, radius, z=0.0):
    """n z-directed unit (1 A m) Hertzian dipoles equally spaced on a horizontal ring."""
    phi = 2.0 * math.pi * np.arange(n) / n
    pos = np.stack([radius * np.cos(phi), radius * np.sin(phi), np.full(n, float(z))], axis=1)
    mom = np.tile(np.array([0.0, 0.0, 1.0]), (n, 1))
    return pos, mom


def body_dipoles():
    """8 z-directed unit dipoles on a 30 cm cylinder at z in {-40,-20,0,20} cm, two azimuths each."""
    pos = []
    for z in (-0.40, -0.20, 0.0, 0.20):
        for phi in (0.0, math.pi):
            pos.append([0.30 * math.cos(phi), 0.30 * math.sin(phi), z])
    pos = np.array(pos)
    return pos, np.tile(np.array([0.0, 0.0, 1.0]), (len(pos), 1))


def inclusion_dipoles():
    """32 z-directed unit dipoles on a 10 cm cylinder: 4 heights x 8 azimuths."""
    pos = []
    for z in (-0.048, -0.016, 0.016, 0.048):
        for k in range(8):
            phi = 2.0 * math.pi * k / 8
            pos.append([0.10 * math.cos(phi), 0.10 * math.sin(phi), z])
    pos = np.array(pos)
    return pos, np.tile(np.array([0.0, 0.0, 1.0]), (len(pos), 1))


def random_coefficients(grid: Grid, nrhs, seed, ncomp=12):
    """Random complex coefficient batch of shape (nrhs, ncomp, Nz, Ny, Nx), entries ~ N(0,1)+iN(0,1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (nrhs, ncomp) + grid.shape
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _head_grid(n):
    h = 0.192 / n
    return Grid(n, n, n, h, h, h)


WORKLOADS = {
    # 16^3 sphere, 12.5 mm voxels, plane wave, one right-hand side
    "sphere16": dict(grid=Grid(16, 16, 16, 0.0125, 0.0125, 0.0125), freq=298e6, source="planewave"),
    # 64^3 head ellipsoid, 3 mm voxels, 16 ring dipoles
    "head64": dict(grid=Grid(64, 64, 64, 0.003, 0.003, 0.003), freq=298e6, source="ring16"),
    # 128 x 128 x 256 body stack, 5 mm voxels, 8 dipoles
    "body128": dict(grid=Grid(128, 128, 256, 0.005, 0.005, 0.005), freq=128e6, source="body8"),
    # 64^3 high-contrast inclusions, 2 mm voxels, 32 dipoles
    "incl64": dict(grid=Grid(64, 64, 64, 0.002, 0.002, 0.002), freq=447e6, source="incl32"),
}


def workload(name, n=None):
    """Materials and sources of a named synthetic workload.

    Returns dict(grid, freq, eps_real, sigma, dip_pos, dip_mom) where dip_* are
    None for the plane-wave case.  `n` overrides the grid size of the head
    workload family (voxel 192 mm / n) used by the serving stream.
    """
    if name == "head" and n is not None:
        g = _head_grid(n)
        eps, sig = head_phantom(g)
        pos, mom = ring_dipoles(16, 0.15)
        return dict(grid=g, freq=298e6, eps_real=eps, sigma=sig, dip_pos=pos, dip_mom=mom)
    w = WORKLOADS[name]
    g = w["grid"]
    if name == "sphere16":
        eps, sig = sphere_phantom(g, 0.1, 50.0, 0.5)
        pos = mom = None
    elif name == "head64":
        eps, sig = head_phantom(g)
        pos, mom = ring_dipoles(16, 0.15)
    elif name == "body128":
        eps, sig = body_phantom(g)
        pos, mom = body_dipoles()
    elif name == "incl64":
        eps, sig = inclusion_phantom(g)
        pos, mom = inclusion_dipoles()
    else:
        raise KeyError(name)
    return dict(grid=g, freq=w["freq"], eps_real=eps, sigma=sig, dip_pos=pos, dip_mom=mom)


def serving_stream(n_requests, seed=77, sizes=(32, 48, 64, 96)):
    """Requests of the serving stream: grid n^3 from `sizes` (voxel 192 mm / n, head phantom with a
    per-request tissue seed), 1..32 z-dipoles on the 15 cm ring, frequency from {64, 128, 298} MHz,
    and unit-rate exponential inter-arrival gaps (scale them by 1/lambda)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n_requests):
        n = int(rng.choice(sizes))
        R = int(rng.integers(1, 33))
        f = float(rng.choice([64e6, 128e6, 298e6]))
        g = _head_grid(n)
        eps, sig = head_phantom(g, seed=int(rng.integers(0, 2**31 - 1)))
        pos, mom = ring_dipoles(R, 0.15)
        out.append(dict(grid=g, freq=f, eps_real=eps, sigma=sig, dip_pos=pos, dip_mom=mom,
                        gap=float(rng.exponential(1.0))))
    return out
