"""Seeded synthetic inputs for the fictitious-wave CSEM hot path.

This module only *describes* problems: node coordinates of the stretched
tensor-product grid, cell resistivities, source / receiver positions,
frequencies and the data-noise recipe.  It holds none of the method's
arithmetic (no spacings, coefficients, time steps or transforms), so that the
CUDA path and the FP64 oracle can both consume it without sharing code.

The marine shapes follow the paper's examples (Sec. 4.2: 0.3 ohm-m water,
1-2.5 ohm-m sediment, a thin 100 ohm-m resistor ~1 km below the seabed,
towed x-dipoles 200-250 m apart, seabed receivers, 0.1-2.25 Hz).  Geometry
conventions: z points down, z = 0 is the top of the grid's core, the CPML is
`npml` cells on every face *outside* the core, stretched cells grow by a fixed
ratio per cell away from the core and CPML cells repeat the last spacing.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


def stretched_axis(h: float, n_core: int, n_lo: int, n_hi: int, n_pml: int,
                   ratio: float, core_start: float) -> np.ndarray:
    """Node coordinates (len = n_pml + n_lo + n_core + n_hi + n_pml + 1).

    The core holds `n_core` cells of width `h` starting at `core_start`.
    Below (above) it `n_lo` (`n_hi`) cells grow by `ratio` per cell outward,
    and `n_pml` cells of the last stretched width pad each end.
    """
    lo = [h * ratio ** (m + 1) for m in range(n_lo)]
    hi = [h * ratio ** (m + 1) for m in range(n_hi)]
    lo += [lo[-1] if lo else h] * n_pml
    hi += [hi[-1] if hi else h] * n_pml
    widths = list(reversed(lo)) + [h] * n_core + hi
    x0 = core_start - sum(lo)
    return x0 + np.concatenate([[0.0], np.cumsum(widths)])


@dataclass
class Points:
    """Point sources or receivers: coordinates (m) and field component (0=x,1=y,2=z)."""
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    comp: np.ndarray

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @staticmethod
    def make(xyz, comp=0) -> "Points":
        a = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
        c = np.full(a.shape[0], comp, dtype=np.int32) if np.isscalar(comp) else np.asarray(comp, np.int32)
        return Points(a[:, 0].copy(), a[:, 1].copy(), a[:, 2].copy(), c)

    def subset(self, idx) -> "Points":
        idx = np.atleast_1d(idx)
        return Points(self.x[idx], self.y[idx], self.z[idx], self.comp[idx])


@dataclass
class Workload:
    name: str
    xn: np.ndarray            # node coordinates (incl. CPML), len nx+1
    yn: np.ndarray
    zn: np.ndarray
    npml: int
    rho: np.ndarray           # current model, cell-centred, shape (nz, ny, nx) [ohm-m]
    rho_true: np.ndarray      # model that generates the observed data
    src: Points
    rec: Points
    freqs: np.ndarray         # Hz
    rho_max: float            # resistivity that freezes the CFL step and CPML d0
    nt: Optional[int] = None  # None -> derived from the slowest decay
    f0: float = 1.0           # reference frequency, omega0 = 2*pi*f0
    precision: int = 32
    kahan: int = 1
    noise: float = 0.0        # relative complex Gaussian noise on observed data
    noise_seed: int = 42
    meta: dict = field(default_factory=dict)

    @property
    def nx(self) -> int:
        return self.xn.size - 1

    @property
    def ny(self) -> int:
        return self.yn.size - 1

    @property
    def nz(self) -> int:
        return self.zn.size - 1

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz


def cell_centres(xn, yn, zn):
    xc = 0.5 * (xn[1:] + xn[:-1])
    yc = 0.5 * (yn[1:] + yn[:-1])
    zc = 0.5 * (zn[1:] + zn[:-1])
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    return X, Y, Z


def layered(xn, yn, zn, water=0.3, seabed=1000.0, sediment=1.0):
    X, Y, Z = cell_centres(xn, yn, zn)
    rho = np.where(Z < seabed, water, sediment).astype(np.float64)
    return rho


def add_slab(rho, xn, yn, zn, half_x=1500.0, half_y=1500.0, top=2000.0, bottom=2050.0, value=100.0):
    X, Y, Z = cell_centres(xn, yn, zn)
    out = rho.copy()
    m = (np.abs(X) <= half_x) & (np.abs(Y) <= half_y) & (Z >= top) & (Z < bottom)
    out[m] = value
    return out


def add_noise(d: np.ndarray, level: float, seed: int) -> np.ndarray:
    """d * (1 + level*(xi1 + i*xi2)/sqrt(2)), xi ~ N(0,1) from default_rng(seed)."""
    if level == 0.0:
        return d.copy()
    rng = np.random.default_rng(seed)
    xi = rng.standard_normal(d.shape) + 1j * rng.standard_normal(d.shape)
    return d * (1.0 + level * xi / np.sqrt(2.0))


# --------------------------------------------------------------------------
# The five marine stand-in workloads
# --------------------------------------------------------------------------

def plain_tiny() -> Workload:
    """Uniform 48^3 core (h=100 m) + 10-cell CPML = 68^3, FP64, 2 layers, 1 dipole, 21 receivers."""
    ax = stretched_axis(100.0, 48, 0, 0, 10, 1.0, 0.0)
    rho = layered(ax, ax, ax, 0.3, 1000.0, 1.0)
    rho_true = layered(ax, ax, ax, 0.3, 1000.0, 2.0)
    src = Points.make([[2400.0, 2400.0, 950.0]], 0)
    rec = Points.make([[x, 2400.0, 1000.0] for x in np.arange(400.0, 4400.0 + 1, 200.0)], 0)
    return Workload("plain_tiny_68c_fp64", ax, ax.copy(), ax.copy(), 10, rho, rho_true, src, rec,
                    np.array([0.25, 0.75]), rho_max=2.0, nt=1500, precision=64, kahan=0)


def thin_reservoir(core_xy=80, core_z=62, n_st_xy=14, n_st_top=6, n_st_bot=8) -> Workload:
    """128x128x96 stretched grid (50 m core cells, ratio 1.05), water/sediment + 100 ohm-m slab."""
    h = 50.0
    xn = stretched_axis(h, core_xy, n_st_xy, n_st_xy, 10, 1.05, -h * core_xy / 2)
    zn = stretched_axis(h, core_z, n_st_top, n_st_bot, 10, 1.05, 0.0)
    rho = layered(xn, xn, zn)
    rho_true = add_slab(rho, xn, xn, zn)
    src = Points.make([[0.0, 0.0, 950.0]], 0)
    rec = Points.make([[x, 0.0, 1000.0] for x in np.arange(-2000.0, 2000.0 + 1, 100.0)], 0)
    return Workload("thin_reservoir_128x128x96_fp32", xn, xn.copy(), zn, 10, rho, rho_true, src, rec,
                    np.array([0.25, 0.5, 0.75, 1.0]), rho_max=100.0, precision=32, kahan=1,
                    noise=0.01, noise_seed=42)


def batched_towline() -> Workload:
    """256x256x128 stretched grid, layered + slab, 32 towline sources, 8x8 seabed receiver array."""
    h = 50.0
    xn = stretched_axis(h, 196, 20, 20, 10, 1.05, -h * 98)
    zn = stretched_axis(h, 94, 6, 8, 10, 1.05, 0.0)
    rho = layered(xn, xn, zn)                      # start model: no reservoir
    rho_true = add_slab(rho, xn, xn, zn)
    src = Points.make([[-3875.0 + 250.0 * i, 0.0, 950.0] for i in range(32)], 0)
    g = np.arange(-1750.0, 1750.0 + 1, 500.0)
    rec = Points.make([[x, y, 1000.0] for y in g for x in g], 0)
    return Workload("batched_towline_256x256x128_32src", xn, xn.copy(), zn, 10, rho, rho_true,
                    src, rec, np.array([0.25, 0.5, 0.75, 1.0]), rho_max=100.0, precision=32, kahan=1)


def large_gradient() -> Workload:
    """400x400x200 stretched grid, 64 sources on two perpendicular towlines, 10x10 receivers, 8 freqs."""
    h = 50.0
    xn = stretched_axis(h, 340, 20, 20, 10, 1.05, -h * 170)
    zn = stretched_axis(h, 166, 6, 8, 10, 1.05, 0.0)
    rho_true = add_slab(layered(xn, xn, zn), xn, xn, zn)
    line = -3875.0 + 250.0 * np.arange(32)
    src = Points.make([[x, 0.0, 950.0] for x in line] + [[0.0, y, 950.0] for y in line], 0)
    g = np.arange(-4500.0, 4500.0 + 1, 1000.0)
    rec = Points.make([[x, y, 1000.0] for y in g for x in g], 0)
    freqs = np.logspace(np.log10(0.1), np.log10(1.5), 8)
    return Workload("large_gradient_400x400x200_64src", xn, xn.copy(), zn, 10, rho_true.copy(), rho_true,
                    src, rec, freqs, rho_max=100.0, precision=32, kahan=1)


def gaussian_random_field(shape, spacing, corr_len, seed):
    """Unit-variance field from FFT-filtered white noise with a Gaussian kernel of length corr_len."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(shape)
    ks = [np.fft.fftfreq(n, d=spacing) * 2 * np.pi for n in shape]
    K2 = sum(k ** 2 for k in np.meshgrid(*ks, indexing="ij"))
    f = np.real(np.fft.ifftn(np.fft.fftn(w) * np.exp(-0.25 * K2 * corr_len ** 2)))
    return (f - f.mean()) / f.std()


def heterogeneous(core_xy=460, core_z=224, n_st=16, n_st_top=6, n_st_bot=6, n_src=16) -> Workload:
    """512x512x256 grid; log10(rho) Gaussian random field below 1 km of 0.3 ohm-m water."""
    h = 50.0
    xn = stretched_axis(h, core_xy, n_st, n_st, 10, 1.05, -h * core_xy / 2)
    zn = stretched_axis(h, core_z, n_st_top, n_st_bot, 10, 1.05, 0.0)
    X, Y, Z = cell_centres(xn, xn, zn)
    grf = gaussian_random_field(Z.shape, h, 500.0, 7)
    rho = np.clip(10.0 ** (0.3 + 0.5 * grf), 0.5, 100.0)
    rho = np.where(Z < 1000.0, 0.3, rho)
    src = Points.make([[-1875.0 + 250.0 * i, 0.0, 950.0] for i in range(n_src)], 0)
    g = np.arange(-1750.0, 1750.0 + 1, 500.0)
    rec = Points.make([[x, y, 1000.0] for y in g for x in g], 0)
    return Workload(f"heterogeneous_{xn.size-1}x{xn.size-1}x{zn.size-1}", xn, xn.copy(), zn, 10, rho, rho,
                    src, rec, np.array([0.25, 0.5, 1.0]), rho_max=100.0, precision=32, kahan=1)


def heterogeneous_crop96() -> Workload:
    """The heterogeneous model cropped to 96^3 cells inside the CPML (116^3 in all), 4 sources."""
    return heterogeneous(core_xy=76, core_z=84, n_st=10, n_st_top=6, n_st_bot=6, n_src=4)


def small_box(n_core=24, h=100.0, npml=8, rho_bg=1.0, layered_model=True, n_freq=2,
              nt=None, n_rec=6, ratio=1.0, n_st=0, n_core_y=None, n_core_z=None) -> Workload:
    """Small seeded test problem spanning a few CUDA tiles with a ragged tail
    (a cube unless n_core_y / n_core_z give other core sizes along y / z)."""
    ncy = n_core if n_core_y is None else n_core_y
    ncz = n_core if n_core_z is None else n_core_z
    xn = stretched_axis(h, n_core, n_st, n_st, npml, ratio, -h * n_core / 2)
    yn = stretched_axis(h, ncy, n_st, n_st, npml, ratio, -h * ncy / 2)
    zn = stretched_axis(h, ncz, n_st, n_st, npml, ratio, 0.0)
    if layered_model:
        seabed = h * (ncz // 3)
        rho = layered(xn, yn, zn, 0.3, seabed, rho_bg)
        rho_true = add_slab(rho, xn, yn, zn, half_x=h * n_core / 5, half_y=h * ncy / 5,
                            top=seabed + 3 * h, bottom=seabed + 4 * h, value=20.0)
        zs = seabed - 0.5 * h
        zr = seabed
    else:
        rho = np.full((zn.size - 1, yn.size - 1, xn.size - 1), rho_bg)
        rho_true = rho * 1.5
        zs = zr = h * ncz / 2
    src = Points.make([[0.3 * h, 0.0, zs]], 0)
    xr = np.linspace(-h * n_core / 3, h * n_core / 3, n_rec)
    rec = Points.make([[x, 0.2 * h, zr] for x in xr], 0)
    freqs = np.array([0.25, 0.75, 1.0, 0.5][:n_freq])
    name = f"small_box_{xn.size-1}c" if (ncy, ncz) == (n_core, n_core) else \
        f"small_box_{xn.size-1}x{yn.size-1}x{zn.size-1}"
    return Workload(name, xn, yn, zn, npml, rho, rho_true, src, rec, freqs,
                    rho_max=float(max(rho.max(), rho_true.max())), nt=nt, precision=32, kahan=1)


ALL = {
    "plain_tiny": plain_tiny,
    "thin_reservoir": thin_reservoir,
    "batched_towline": batched_towline,
    "large_gradient": large_gradient,
    "heterogeneous": heterogeneous,
    "heterogeneous_crop96": heterogeneous_crop96,
}
