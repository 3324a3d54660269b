"""Seeded, synthetic inputs for the string method: initial paths and the benchmark workloads.

This module builds inputs only; it holds none of the method's arithmetic (no field, step, energy or
reparametrisation) and is the one module that both the CUDA path's callers and the CPU oracle's
callers draw their inputs from.

Initial paths (Sec. IV): a radially symmetric Neel skyrmion with the linear polar profile
theta(r) = pi (1 - r/R) for r < R (core down, s_z = -1 at the centre) in a +z background, the same
in every z layer (a cylinder), and the +z ferromagnet as the last image.
  * Bloch-point path: image k scales the polar angle by (1 - k/(K-1)), so the skyrmion shrinks into
    the ferromagnet.
  * boundary path: image k shifts the skyrmion centre along +x from the lattice centre to R past
    the last column, so the skyrmion leaves through the edge; the last image is exactly +z.
Helicity: psi = pi for D > 0 and psi = 0 for D < 0 (the sign that makes the DMI energy of Eq. 1
negative for a Neel skyrmion).

Layout of every returned array: float64 ``[image][site][3]`` (or ``[site][3]``), site index
``(z*ny + y)*nx + x``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def _polar_field(nx, ny, nz, theta, phi):
    s = np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)], axis=-1)
    s = np.broadcast_to(s[None], (nz, ny, nx, 3))
    return np.ascontiguousarray(s.reshape(nz * ny * nx, 3))


def helicity(D: float) -> float:
    return math.pi if D > 0 else 0.0


def skyrmion_angles(nx, ny, R, xc=None, yc=None, psi=math.pi, theta_scale=1.0):
    """Polar and azimuthal angle fields [ny, nx] of a Neel skyrmion centred at (xc, yc)."""
    xc = (nx - 1) / 2.0 if xc is None else xc
    yc = (ny - 1) / 2.0 if yc is None else yc
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    r = np.sqrt((x - xc) ** 2 + (y - yc) ** 2)
    theta = np.where(r < R, math.pi * (1.0 - r / R), 0.0) * theta_scale
    phi = np.arctan2(y - yc, x - xc) + psi
    return theta, phi


def skyrmion(nx, ny, nz, R, D=1.0, xc=None, yc=None) -> np.ndarray:
    theta, phi = skyrmion_angles(nx, ny, R, xc, yc, helicity(D))
    return _polar_field(nx, ny, nz, theta, phi)


def ferromagnet(nx, ny, nz) -> np.ndarray:
    s = np.zeros((nx * ny * nz, 3))
    s[:, 2] = 1.0
    return s


def bloch_point_path(nx, ny, nz, n_images, R, D=1.0) -> np.ndarray:
    out = np.empty((n_images, nx * ny * nz, 3))
    for k in range(n_images):
        theta, phi = skyrmion_angles(nx, ny, R, psi=helicity(D), theta_scale=1.0 - k / (n_images - 1))
        out[k] = _polar_field(nx, ny, nz, theta, phi)
    return out


def boundary_path(nx, ny, nz, n_images, R, D=1.0) -> np.ndarray:
    out = np.empty((n_images, nx * ny * nz, 3))
    x0, x1 = (nx - 1) / 2.0, (nx - 1) + R
    for k in range(n_images):
        if k == n_images - 1:
            out[k] = ferromagnet(nx, ny, nz)
            continue
        xc = x0 + (x1 - x0) * k / (n_images - 1)
        theta, phi = skyrmion_angles(nx, ny, R, xc=xc, psi=helicity(D))
        out[k] = _polar_field(nx, ny, nz, theta, phi)
    return out


def random_spins(shape, seed: int) -> np.ndarray:
    """Random unit vectors (Gaussian direction), float64, last axis 3."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(tuple(shape))
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def crop(path, nx, ny, nz, x0, x1, y0, y1, z0, z1) -> np.ndarray:
    """Sub-lattice [x0,x1) x [y0,y1) x [z0,z1) of a [K, N, 3] path."""
    K = path.shape[0]
    p = path.reshape(K, nz, ny, nx, 3)[:, z0:z1, y0:y1, x0:x1]
    return np.ascontiguousarray(p.reshape(K, -1, 3))


@dataclasses.dataclass(frozen=True)
class StringSpec:
    nx: int
    ny: int
    nz: int
    J: float
    D: float
    K: float
    w: float
    n_images: int
    path: str      # "bloch" or "boundary"
    R: float

    @property
    def n_sites(self) -> int:
        return self.nx * self.ny * self.nz

    def initial_path(self) -> np.ndarray:
        if self.path == "bloch":
            return bloch_point_path(self.nx, self.ny, self.nz, self.n_images, self.R, self.D)
        return boundary_path(self.nx, self.ny, self.nz, self.n_images, self.R, self.D)


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    strings: tuple
    n_iter: int
    dt: float = 0.1

    @property
    def spin_updates_per_iter(self) -> int:
        return sum(s.n_sites * s.n_images for s in self.strings)


def tiny_bloch() -> Workload:
    """16x16x1, 16 images, J=1 D=0.3 K=0.05 w=0.01, R=4 Bloch-point path, 200 iterations."""
    return Workload("tiny-16x16x1-K16", (StringSpec(16, 16, 1, 1.0, 0.3, 0.05, 0.01, 16, "bloch", 4.0),), 200)


def bloch_collapse() -> Workload:
    """64x64x8 cylinder skyrmion (R=8) to ferromagnet, 32 images, D=0.25 K=0.1 w=0.02, 2000 iterations."""
    return Workload("bloch-64x64x8-K32", (StringSpec(64, 64, 8, 1.0, 0.25, 0.1, 0.02, 32, "bloch", 8.0),), 2000)


def bloch_collapse_crop_path(path64: np.ndarray) -> np.ndarray:
    """The 16x16x4 crop (x, y in [24, 40), z in [2, 6)) of a 64x64x8 path."""
    return crop(path64, 64, 64, 8, 24, 40, 24, 40, 2, 6)


def boundary_sweep() -> Workload:
    """128x128x4, R=10 edge paths, 48 images, 8 (K, D) points, w=0.01, 2000 iterations."""
    strings = tuple(StringSpec(128, 128, 4, 1.0, D, K, 0.01, 48, "boundary", 10.0)
                    for K in (0.0, 0.05, 0.1, 0.2) for D in (0.2, 0.35))
    return Workload("boundary-sweep-128x128x4-8x48", strings, 2000)


def uneven_study(seed: int = 7) -> Workload:
    """20 strings x 32 images; sizes from {64^2x4, 96^2x4, 128^2x8, 192^2x8}, K~U[0,0.2], D~U[0.15,0.4];
    draws in the order (size index, K, D) per string; R = nx/8; Bloch path for even strings, boundary
    path for odd ones; w = 0.01; 5000 iterations."""
    sizes = ((64, 4), (96, 4), (128, 8), (192, 8))
    rng = np.random.default_rng(seed)
    strings = []
    for i in range(20):
        si = int(rng.integers(0, len(sizes)))
        K = float(rng.uniform(0.0, 0.2))
        D = float(rng.uniform(0.15, 0.4))
        n, nz = sizes[si]
        strings.append(StringSpec(n, n, nz, 1.0, D, K, 0.01, 32, "bloch" if i % 2 == 0 else "boundary", n / 8.0))
    return Workload("uneven-study-20x32", tuple(strings), 5000)


# ---- the paper's monolayer (Sec. IV) ------------------------------------------------------------------
# 112 x 112 x 1 sites on a simple cubic lattice, a = 0.2715 nm, |S| = 2.3737 mu_B, J = 54.23 meV, 60 images
# per string; the DM and anisotropy energies d and k are varied.  In the library's reduced units energies
# are in J: D = d / J, K = k / J and w = mu0 |S|^2 / (4 pi a^3) / J.
PAPER_A_NM = 0.2715
PAPER_MOMENT_MUB = 2.3737
PAPER_J_MEV = 54.23
MU0 = 1.25663706212e-6          # vacuum permeability, N / A^2 (CODATA 2018)
MU_B = 9.2740100783e-24         # Bohr magneton, J / T (CODATA 2018)
MEV = 1.602176634e-22           # 1 meV in J (exact)


def paper_w() -> float:
    """Reduced dipole strength w / J of the paper's constants (about 2.79e-4)."""
    S = PAPER_MOMENT_MUB * MU_B
    a = PAPER_A_NM * 1e-9
    return MU0 * S * S / (4.0 * math.pi * a ** 3) / (PAPER_J_MEV * MEV)


def paper_monolayer(d_meV: float = 5.30, k_meV: float = 1.0, path: str = "bloch", n_images: int = 60) -> StringSpec:
    """One string of the paper's monolayer: d and k in meV; initial skyrmion radius 14 sites (nx/8)."""
    return StringSpec(112, 112, 1, 1.0, d_meV / PAPER_J_MEV, k_meV / PAPER_J_MEV, paper_w(), n_images, path, 14.0)


def paper_monolayer_workload() -> Workload:
    """The paper's monolayer at d = 5.30 meV (its Fig. 4 value), k = 1.0 meV, Bloch-point path, 5000
    iterations (the paper runs 100-10000)."""
    return Workload("paper-monolayer-112x112x1-K60", (paper_monolayer(),), 5000)


PHASE_D_MEV = (4.5, 5.3, 6.1)
PHASE_K_MEV = (0.8, 1.2, 1.6)


def paper_phase_diagram() -> Workload:
    """A 3 x 3 (d, k) grid in meV around the paper's d = 5.30 meV, for both annihilation paths (18 strings
    of 60 images on the 112 x 112 x 1 monolayer), 5000 iterations."""
    strings = tuple(paper_monolayer(d, k, path) for path in ("bloch", "boundary") for d in PHASE_D_MEV for k in PHASE_K_MEV)
    return Workload("paper-phase-diagram-112x112x1-18x60", strings, 5000)

