"""Seeded synthetic inputs for the BdG eigensolver workloads.

This module only draws random numbers and lays out fields on the grid; it
holds none of the eigensolver's arithmetic.  Both the FP64 CPU oracle and the
CUDA library consume what it returns, so the two sides always see the same
bytes.

Conventions (shared by every consumer):
  * grid Nx x Ny x Nz, spacing dx = 1, periodic (paper, "Numerical setup and
    implementation");
  * site index s = (ix*Ny + iy)*Nz + iz (z fastest);
  * coordinates x = ix - Nx/2 (likewise y, z) so the box centre is a site;
  * U is a real float64 array of length V = Nx*Ny*Nz, Delta a complex128
    array of length V; the BdG matrix has dimension N = 2V.

Recipe for the random fields:
  smooth field: white N(0,1) on the grid -> FFT -> multiply by
  exp(-|k|^2 l^2 / 4) -> inverse FFT -> real part -> normalise to unit
  standard deviation -> scale by the amplitude.
  vortex pairing field: Delta = A * prod_j tanh(rho_j / 2) * exp(i sum_j s_j phi_j)
  with minimum-image distances rho_j to straight z-lines and phi_j the
  azimuth about line j (phi = 0 on the line itself).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Workload", "coords", "smooth_field", "vortex_pairing", "uniform",
    "random_small", "c1_uniform", "c2_single_vortex", "c3_vortex_lattice",
    "c4_tubes", "c5_sample", "c5_small_sample", "by_name", "unit_vectors",
]


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    mu: float
    U: np.ndarray          # float64, length V
    Delta: np.ndarray      # complex128, length V
    meta: dict = field(default_factory=dict)

    @property
    def V(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def N(self) -> int:
        return 2 * self.V


def coords(nx: int, ny: int, nz: int):
    """Site coordinates x, y, z (each float64, length V) in z-fastest order."""
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    return ((ix - nx // 2).ravel().astype(np.float64),
            (iy - ny // 2).ravel().astype(np.float64),
            (iz - nz // 2).ravel().astype(np.float64))


def smooth_field(shape, ell: float, seed: int, amplitude: float) -> np.ndarray:
    """Seeded Gaussian random field with correlation length ell (flattened)."""
    rng = np.random.default_rng(seed)
    white = rng.standard_normal(shape)
    ks = [2 * np.pi * np.fft.fftfreq(n) for n in shape]
    kk = np.meshgrid(*ks, indexing="ij")
    k2 = sum(k * k for k in kk)
    f = np.fft.ifftn(np.fft.fftn(white) * np.exp(-k2 * ell * ell / 4.0)).real
    f = (f - f.mean()) / f.std()
    return (amplitude * f).ravel()


def vortex_pairing(nx, ny, nz, amplitude, centers, charges) -> np.ndarray:
    """Straight z-vortices at (xc, yc) with winding numbers `charges`."""
    x, y, _ = coords(nx, ny, nz)
    mag = np.full(x.shape, float(amplitude))
    phase = np.zeros(x.shape)
    for (xc, yc), s in zip(centers, charges):
        dx = (x - xc + nx / 2.0) % nx - nx / 2.0
        dy = (y - yc + ny / 2.0) % ny - ny / 2.0
        rho = np.hypot(dx, dy)
        mag = mag * np.tanh(rho / 2.0)
        phase = phase + s * np.arctan2(dy, dx)
    return mag * np.exp(1j * phase)


def uniform(nx, ny, nz, mu=0.5, U0=0.0, Delta0=0.2, name="uniform") -> Workload:
    V = nx * ny * nz
    return Workload(name, nx, ny, nz, mu, np.full(V, float(U0)),
                    np.full(V, complex(Delta0), dtype=np.complex128),
                    {"kind": "uniform", "U0": U0, "Delta0": Delta0})


def random_small(nx, ny, nz, seed=0, mu=0.5, amplitude=0.3, n_vortices=1,
                 U0=-0.4, U_amp=0.05, ell=2.0, name=None) -> Workload:
    """Small inhomogeneous case (vortices + smooth random U) for parity tests."""
    rng = np.random.default_rng(10_000 + seed)
    centers = [(rng.uniform(-nx / 2, nx / 2), rng.uniform(-ny / 2, ny / 2))
               for _ in range(n_vortices)]
    charges = [1 if i % 2 == 0 else -1 for i in range(n_vortices)]
    D = vortex_pairing(nx, ny, nz, amplitude, centers, charges)
    U = U0 + smooth_field((nx, ny, nz), ell, seed, U_amp)
    return Workload(name or f"random_{nx}x{ny}x{nz}_s{seed}", nx, ny, nz, mu, U, D,
                    {"kind": "random_small", "seed": seed, "centers": centers})


def c1_uniform() -> Workload:
    """Uniform periodic 8x8x8, mu=0.5, U=0, Delta=0.2 (N=1024)."""
    w = uniform(8, 8, 8, 0.5, 0.0, 0.2, name="C1_uniform_8x8x8")
    return w


def c2_single_vortex() -> Workload:
    """16^3, one vortex on the z axis through x=y=0, |Delta|=0.3, U=-0.4+0.05*field (N=8192)."""
    nx = ny = nz = 16
    D = vortex_pairing(nx, ny, nz, 0.3, [(0.0, 0.0)], [1])
    U = -0.4 + smooth_field((nx, ny, nz), 3.0, 1, 0.05)
    return Workload("C2_single_vortex_16x16x16", nx, ny, nz, 0.5, U, D,
                    {"kind": "vortex", "centers": [(0.0, 0.0)]})


def _vortex_positions(nx, ny, count, seed, min_sep):
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < count:
        p = (rng.uniform(-nx / 2, nx / 2), rng.uniform(-ny / 2, ny / 2))
        ok = True
        for q in pts:
            dx = (p[0] - q[0] + nx / 2) % nx - nx / 2
            dy = (p[1] - q[1] + ny / 2) % ny - ny / 2
            if math.hypot(dx, dy) < min_sep:
                ok = False
                break
        if ok:
            pts.append(p)
    return pts


def c3_vortex_lattice() -> Workload:
    """24x24x32, four z-vortices (+1,-1,+1,-1), |Delta|=0.25, U=-0.4+0.05*field (N=36864)."""
    nx, ny, nz = 24, 24, 32
    centers = _vortex_positions(nx, ny, 4, 2, 6.0)
    D = vortex_pairing(nx, ny, nz, 0.25, centers, [1, -1, 1, -1])
    U = -0.4 + smooth_field((nx, ny, nz), 3.0, 3, 0.05)
    return Workload("C3_vortex_lattice_24x24x32", nx, ny, nz, 0.5, U, D,
                    {"kind": "vortex", "centers": centers})


def c4_tubes(sizes=(16, 24, 32, 48), nz=64):
    """Tube cross-sections Nx=Ny=L with kz conserved: (L, U2d, Delta2d, kz list).

    Each geometry carries one vortex on its axis and a seeded 2-D U field
    (seed 4+i).  The kz values are 2*pi*n/nz for n = -nz/2 .. nz/2-1, one BdG
    block of size 2*L*L per kz.
    """
    out = []
    for i, L in enumerate(sizes):
        D = vortex_pairing(L, L, 1, 0.3, [(0.0, 0.0)], [1])
        U = -0.4 + smooth_field((L, L), 3.0, 4 + i, 0.05)
        kz = [2 * np.pi * n / nz for n in range(-nz // 2, nz // 2)]
        out.append({"L": L, "mu": 0.5, "U": U, "Delta": D, "kz": kz})
    return out


def c5_sample(seed: int, n=24, min_sep=4.0) -> Workload:
    """One seeded learned-guess sample on n^3: mu, target gap, 0-4 straight vortices."""
    rng = np.random.default_rng(50_000 + seed)
    mu = rng.uniform(0.3, 0.7)
    d0 = rng.uniform(0.1, 0.4)
    nv = int(rng.integers(0, 5))
    centers = _vortex_positions(n, n, nv, 60_000 + seed, min_sep) if nv else []
    charges = [1 if i % 2 == 0 else -1 for i in range(nv)]
    D = vortex_pairing(n, n, n, d0, centers, charges)
    U = np.zeros(n ** 3)
    return Workload(f"C5_sample_{seed}", n, n, n, mu, U, D,
                    {"kind": "learned", "Delta0": d0, "centers": centers})


def c5_small_sample(seed: int, n=8) -> Workload:
    """Learned-guess sample for small boxes (n^3 with n < 16, where the gap range of the full
    recipe gives a coherence length beyond the box): mu ~ U[0.45, 0.6], Delta0 ~ U[0.4, 0.5],
    no vortex or one straight z-vortex at a seeded position."""
    rng = np.random.default_rng(70_000 + seed)
    mu = rng.uniform(0.45, 0.6)
    d0 = rng.uniform(0.4, 0.5)
    nv = int(rng.integers(0, 2))
    centers = [(rng.uniform(-n / 2, n / 2), rng.uniform(-n / 2, n / 2))] if nv else []
    D = vortex_pairing(n, n, n, d0, centers, [1] * nv)
    return Workload(f"C5_small_sample_{seed}", n, n, n, mu, np.zeros(n ** 3), D,
                    {"kind": "learned", "Delta0": d0, "centers": centers})


def by_name(name: str) -> Workload:
    return {"C1": c1_uniform, "C2": c2_single_vortex, "C3": c3_vortex_lattice}[name]()


def unit_vectors(n: int, ncols: int, seed: int) -> np.ndarray:
    """Seeded random complex unit columns (n x ncols, column-major-friendly)."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, ncols)) + 1j * rng.standard_normal((n, ncols))
    return X / np.linalg.norm(X, axis=0, keepdims=True)
