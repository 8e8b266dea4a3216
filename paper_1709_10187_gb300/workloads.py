"""Seeded synthetic workloads (grids, media, sources) shared by the tests, the
benchmark, the CUDA path and the CPU oracle.

This module only *describes inputs*: grid sizes, frequency edges, densities,
velocities and seeds.  It holds none of the method's arithmetic (no opacities,
leakage coefficients or random walks), so both implementations may use it.

Slab workloads follow Sec. 3.2 / Sec. 4.2 of Smith et al. (2017): a uniform,
static, isothermal slab |z| <= R with a monochromatic line-centre source at the
midplane.  P1 is the setup of Fig. 2 (a tau0 = 1e9, T = 10 K,
dz ~ 0.01 R, dx ~ 0.05 (a tau0)^(1/3) over |x| <= 2.5 (a tau0)^(1/3)); P2 is the
coarser matched resolution n_z = 101, n_x = 51 suggested in Sec. 4.2.
"""
from __future__ import annotations

import dataclasses
from typing import Optional, Tuple

import numpy as np

GEOM_SLAB_1D = 1
GEOM_CART_3D = 3


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    ndim: int                 # 1 = slab along one axis, 3 = Cartesian cube
    n: Tuple[int, int, int]   # cells per axis (unused axes 1)
    J: int                    # frequency bins
    x_min: float              # comoving frequency range in Doppler widths
    x_max: float
    tau0: float               # k0 * R at unit density (line-centre optical depth)
    T: float                  # K, isothermal
    packets: int
    seed: int
    R: float = 1.0
    x0: float = 0.0           # source frequency
    sphere: bool = False      # 3D: medium only in cells whose centre has r < R
    vmax_kms: float = 0.0     # 3D Hubble-like outflow v = vmax * r / R
    atau0_nominal: Optional[float] = None  # the a*tau0 the config is quoted at
    core_half: float = 0.0    # > 0: one central bin [-core_half, core_half], unit-width wing bins

    @property
    def ncell(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    def edges(self) -> np.ndarray:
        """J+1 bin edges (float64): uniform over [x_min, x_max], or with
        core_half > 0 the wide-core grid of wide_core_edges(x_max, core_half)."""
        if self.core_half > 0.0:
            e = wide_core_edges(self.x_max, self.core_half)
            if len(e) != self.J + 1 or e[0] != self.x_min:
                raise ValueError(f"{self.name}: J / x_min do not match the wide-core grid ({len(e) - 1} bins)")
            return e
        return np.linspace(self.x_min, self.x_max, self.J + 1, dtype=np.float64)

    def cell_centres(self) -> np.ndarray:
        """Cell-centre coordinates, shape (ncell, 3), axis 0 fastest; unused axes 0."""
        axes = []
        for a in range(3):
            if a < self.ndim:
                m = self.n[a]
                axes.append(-self.R + (np.arange(m) + 0.5) * (2.0 * self.R / m))
            else:
                axes.append(np.zeros(1))
        z, y, x = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
        return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)

    def mask(self) -> Optional[np.ndarray]:
        """uint8 medium mask (1 = medium, 0 = vacuum), or None for a full grid."""
        if not self.sphere:
            return None
        r = np.linalg.norm(self.cell_centres(), axis=1)
        return (r < self.R).astype(np.uint8)

    def velocity_kms(self) -> Optional[np.ndarray]:
        """Per-cell bulk velocity in km/s, shape (ncell, 3), or None if static."""
        if self.vmax_kms == 0.0:
            return None
        return (self.vmax_kms * self.cell_centres() / self.R).astype(np.float64)

    def with_(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


def wide_core_edges(x_max: float, core_half: float, dx: float = 1.0) -> np.ndarray:
    """Frequency edges with the resolution Sec. 5.1 suggests: one central bin
    [-core_half, core_half] at least 2 x_cw wide (an effective core-skipping
    scheme) and wing bins dx wide out to the last edge <= x_max."""
    k = int(np.floor((x_max - core_half) / dx + 1e-9))
    wing = core_half + dx * np.arange(1, k + 1)
    return np.concatenate([-wing[::-1], [-core_half, core_half], wing]).astype(np.float64)


# k0 R for a tau0 = 1e9 at T = 10 K: a(10 K) = 4.702e-4 * (1e-3)^(-1/2) = 1.48691e-2.
_TAU0_ATAU1E9_T10 = 6.725395e10

C1 = Workload("slab_tau1e5_64x128", 1, (64, 1, 1), 128, -30.0, 30.0, 1.0e5, 1.0e4, 100_000, 0x5EED0001)
C2 = Workload("slab_tau1e7_256x512", 1, (256, 1, 1), 512, -60.0, 60.0, 1.0e7, 1.0e4, 10_000_000, 0x5EED0002)
# C2 on the wide-core grid: central bin +-3.3 (x_cw = 3.255 at 1e4 K), unit wing bins to +-59.3 (113 bins)
C2_WIDECORE = Workload("slab_tau1e7_256x113_widecore", 1, (256, 1, 1), 113, -59.3, 59.3, 1.0e7, 1.0e4, 10_000_000,
                       0x5EED0012, core_half=3.3)
C1_WIDECORE = Workload("slab_tau1e5_64x53_widecore", 1, (64, 1, 1), 53, -29.3, 29.3, 1.0e5, 1.0e4, 100_000,
                       0x5EED0011, core_half=3.3)
P1 = Workload("slab_atau1e9_T10_201x101", 1, (201, 1, 1), 101, -2500.0, 2500.0, _TAU0_ATAU1E9_T10, 10.0,
              1_000_000, 0x5EED0011, atau0_nominal=1.0e9)
P2 = Workload("slab_atau1e9_T10_101x51", 1, (101, 1, 1), 51, -2500.0, 2500.0, _TAU0_ATAU1E9_T10, 10.0,
              1_000_000, 0x5EED0012, atau0_nominal=1.0e9)
C3 = Workload("sphere_tau1e7_64c_128b", 3, (64, 64, 64), 128, -80.0, 80.0, 1.0e7, 1.0e4, 10_000_000,
              0x5EED0003, sphere=True)

C3_V20 = C3.with_(name="sphere_tau1e7_64c_128b_v20", vmax_kms=20.0)
C3_V200 = C3.with_(name="sphere_tau1e7_64c_128b_v200", vmax_kms=200.0)

# The grey diffusion test (Sec. 3): 101 cells, one frequency bin, so every state
# has the same opacity and the walk is spatial diffusion with D = 1/(3k).
GREY101 = Workload("grey_slab_101x1", 1, (101, 1, 1), 1, -5.0, 5.0, 1.0e3, 1.0e4, 10_000_000, 0x5EED0901)

# Small grids for parity tests: several row tiles and ragged sizes, cheap enough
# for the oracle to finish in seconds.
TINY = Workload("slab_tiny_8x16", 1, (8, 1, 1), 16, -8.0, 8.0, 2.0e2, 1.0e4, 20_000, 0x5EED0101)
SMALL = Workload("slab_small_13x37", 1, (13, 1, 1), 37, -12.0, 12.0, 1.0e3, 1.0e4, 20_000, 0x5EED0102)
GREY_LIKE = Workload("slab_wide_bins_31x9", 1, (31, 1, 1), 9, -90.0, 90.0, 3.0e4, 1.0e4, 20_000, 0x5EED0103)

# 3D spheres small enough for the exact chain: cube of 8^3 cells, medium where
# the cell centre is inside r < R, static or in Hubble-like outflow.
SPHERE8 = Workload("sphere_tiny_8c_16b", 3, (8, 8, 8), 16, -16.0, 16.0, 1.0e3, 1.0e4, 20_000, 0x5EED0301, sphere=True)
SPHERE8_V = SPHERE8.with_(name="sphere_tiny_8c_16b_v20", vmax_kms=20.0, seed=0x5EED0302)
SPHERE9_V = Workload("sphere_small_9c_21b_v20", 3, (9, 9, 9), 21, -21.0, 21.0, 3.0e3, 1.0e4, 10_000, 0x5EED0303,
                     sphere=True, vmax_kms=20.0)

ALL = {w.name: w for w in (C1, C2, C1_WIDECORE, C2_WIDECORE, P1, P2, C3, C3_V20, C3_V200, GREY101, TINY, SMALL,
                           GREY_LIKE, SPHERE8, SPHERE8_V, SPHERE9_V)}


def time_edges(dt: float, t_end: float) -> np.ndarray:
    """Edges 0, dt, 2 dt, ... of constant time steps up to t_end (in R/c)."""
    n = int(round(t_end / dt))
    return np.arange(n + 1, dtype=np.float64) * dt


def batched_instances(n: int = 512, seed: int = 0x5EED0004, packet_scale: float = 1.0):
    """The batched workload: n independent slab or sphere instances (p = 1/2),
    tau0 log-uniform in [1e4, 1e8], T log-uniform in [1e2, 1e5] K, cells
    uniform in {32..256} (a sphere takes the nearest integer cube root per
    axis), 128-512 bins, packets log-uniform in [1e4, 1e6] (times
    packet_scale).  Each instance's frequency grid covers
    |x| <= max(4 (a tau0)^(1/3), bins/2), with a = 4.702e-4 (T/1e4 K)^(-1/2) the
    damping parameter, i.e. bins at least one Doppler width wide and the escape
    peaks (~(a tau0)^(1/3)) inside the grid."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        sphere = bool(rng.random() < 0.5)
        tau0 = float(10 ** rng.uniform(4, 8))
        T = float(10 ** rng.uniform(2, 5))
        cells = int(rng.integers(32, 257))
        J = int(rng.integers(128, 513))
        npk = max(1, int(round(packet_scale * 10 ** rng.uniform(4, 6))))
        atau = 4.702e-4 / np.sqrt(T / 1.0e4) * tau0
        xmax = float(max(4.0 * atau ** (1.0 / 3.0), J / 2.0))
        if sphere:
            m = max(2, int(round(cells ** (1.0 / 3.0))))
            w = Workload(f"batch{i}_sphere", 3, (m, m, m), J, -xmax, xmax, tau0, T, npk, seed + i, sphere=True)
        else:
            w = Workload(f"batch{i}_slab", 1, (cells, 1, 1), J, -xmax, xmax, tau0, T, npk, seed + i)
        out.append(w)
    return out


def gaussian_random_field(n: int, slope: float, rng) -> np.ndarray:
    """Zero-mean, unit-variance Gaussian random field on an n^3 periodic grid
    with power spectrum P(k) ~ k^slope (FFT of white noise shaped by
    k^(slope/2); the k = 0 mode is dropped)."""
    noise = rng.standard_normal((n, n, n))
    fk = np.fft.rfftn(noise)
    kx = np.fft.fftfreq(n)[:, None, None]
    ky = np.fft.fftfreq(n)[None, :, None]
    kz = np.fft.rfftfreq(n)[None, None, :]
    k = np.sqrt(kx * kx + ky * ky + kz * kz)
    amp = np.zeros_like(k)
    amp[k > 0] = k[k > 0] ** (slope / 2.0)
    g = np.fft.irfftn(fk * amp, s=(n, n, n), axes=(0, 1, 2))
    g -= g.mean()
    return g / g.std()


@dataclasses.dataclass(frozen=True)
class ClumpyMedium:
    """Brick-resolution clumpy medium: a lognormal density and a Gaussian
    turbulent velocity, constant over bricks of `brick`^3 cells whose
    boundaries sit at cell indices = offset (mod brick) on every axis (partial
    bricks at the cube's faces when offset > 0)."""
    workload: Workload
    brick: int
    n_rel: np.ndarray   # per cell, axis 0 fastest (mean 1)
    v_kms: np.ndarray   # per cell x3
    brick_rho: np.ndarray  # per brick (nbx^3, axis 0 fastest)
    offset: int = 0
    nbx: int = 0        # bricks per axis, partial ones included
    full: np.ndarray = None  # per brick: True when all brick^3 cells lie in the cube


def brick_lattice(n: int, brick: int, offset: int):
    """Bricks per axis and the brick coordinate of every cell index along an
    axis of n cells for a lattice of `brick`-cell bricks with a boundary at
    cell index `offset`."""
    sh = (brick - offset % brick) % brick
    nbx = (n + sh + brick - 1) // brick
    c = (np.arange(n) + sh) // brick
    return nbx, c, sh


def clumpy_medium(n: int = 128, J: int = 256, x_max: float = 256.0, tau0: float = 1.0e7, T: float = 1.0e4,
                  brick: int = 8, sigma_ln: float = 1.0, slope: float = -11.0 / 3.0, sigma_v_kms: float = 10.0,
                  packets: int = 100_000_000, seed: int = 0x5EED0005, name: str = "clumpy",
                  offset: int = 0) -> ClumpyMedium:
    """The clumpy 3D workload: an n^3 cube of cells x J bins over [-x_max, x_max],
    lognormal density rho = exp(sigma_ln g - sigma_ln^2/2) from a Gaussian
    random field g with spectral slope `slope`, three independent fields of the
    same spectrum for the velocity (sigma_v per component), both drawn on the
    grid of bricks and held constant inside each brick; tau0 is the line-centre
    optical depth centre-to-face at the mean density.  The brick boundaries sit
    at cell indices = offset (mod brick); with offset 0 and n a multiple of
    brick every brick is whole."""
    rng = np.random.default_rng(seed)
    nbx, c, sh = brick_lattice(n, brick, offset)
    g = gaussian_random_field(nbx, slope, rng)
    rho_b = np.exp(sigma_ln * g - 0.5 * sigma_ln ** 2)
    v_b = np.stack([sigma_v_kms * gaussian_random_field(nbx, slope, rng) for _ in range(3)], axis=-1)
    # (i2, i1, i0) index order of the brick fields -> per-cell arrays, axis 0 fastest
    rep = lambda a: a[np.ix_(c, c, c)]
    rho_c = rep(rho_b)
    v_c = np.stack([rep(v_b[..., a]) for a in range(3)], axis=-1)
    lo = np.arange(nbx) * brick - sh
    full1 = (lo >= 0) & (lo + brick <= n)
    full = full1[:, None, None] & full1[None, :, None] & full1[None, None, :]
    w = Workload(name, 3, (n, n, n), J, -x_max, x_max, tau0, T, packets, seed)
    return ClumpyMedium(w, brick, rho_c.reshape(-1).astype(np.float64), v_c.reshape(-1, 3).astype(np.float64),
                        rho_b.reshape(-1).astype(np.float64), offset, nbx, full.reshape(-1))
