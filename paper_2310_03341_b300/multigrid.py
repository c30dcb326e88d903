"""Multigrid start of the self-consistent loop: the static solution is converged first on coarser
lattices of the same box, and each converged solution, interpolated spectrally, starts the loop on
the next finer lattice (paper, "Performance of the Matrix Diagonalization Algorithm": lattices of
60, 80 and 100 points per direction at a fixed domain size).

Lattices of spacing dx on the unit-spacing library.  The kinetic operator on spacing dx is the
unit-spacing one divided by dx^2, so with s = dx^2

    H_dx(mu, U, Delta) = H_1(s mu, s U, s Delta) / s:

the eigenvectors are those of the scaled unit-spacing problem and the eigenvalues are divided by
s.  The lattice cutoff pi^2 / (2 dx^2) becomes pi^2 / 2, the densities per unit volume are the
per-site densities divided by dx^3, and the contact update Delta = g nu, U = -g n / 2 becomes the
unit-spacing update with the coupling g / dx.  Every level therefore runs the ordinary loop
(bdg_scf_step on a grid of unit spacing) in scaled units.  Its coupling comes from that level's own
uniform gap equation (the same Delta0 at the same mu), so each level has its own coupling and its own
uniform Hartree shift U0.  What passes from level to level is the deviation from the uniform state,
U - U0, and the signed pairing amplitude A = Re(Delta e^{-i theta}) along the fixed vortex phase,
both in physical units.

Geometry.  A level with n points per direction has spacing L / n in the box of the finest level
(L = its point count, spacing 1).  The site (i - n/2) dx is the physical coordinate, so the box
centre is a site on every level, and index 0 sits at -L/2 on every level.  Every direction is
scaled by the same ratio, and each level's point counts must be even.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time
from dataclasses import dataclass

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def level_shape(shape, ratio: float):
    """Point counts of the level that has `ratio` times the points of `shape` per direction."""
    out = []
    for n in shape:
        m = n * ratio
        if abs(m - round(m)) > 1e-9 or int(round(m)) < 2 or int(round(m)) % 2:
            raise ValueError(f"ratio {ratio} gives {m} points for {n}: every level needs even counts >= 2")
        out.append(int(round(m)))
    return tuple(out)


def _upsample_axis(F, nc: int, nf: int, axis: int):
    """Zero-pad the DFT coefficients of one axis from nc to nf modes.  The modes m keep their
    wavenumbers 2 pi m / L; the Nyquist mode m = -nc/2 is split evenly between -nc/2 and +nc/2,
    so that a real field stays real."""
    if nf == nc:
        return F
    shape = list(F.shape)
    shape[axis] = nf
    G = np.zeros(shape, dtype=np.complex128)
    h = nc // 2

    def sl(a, b):
        idx = [slice(None)] * F.ndim
        idx[axis] = slice(a, b)
        return tuple(idx)

    G[sl(0, h)] = F[sl(0, h)]                          # m = 0 .. nc/2 - 1
    G[sl(nf - h + 1, nf)] = F[sl(h + 1, nc)]           # m = -nc/2 + 1 .. -1
    G[sl(h, h + 1)] += 0.5 * F[sl(h, h + 1)]           # Nyquist, +nc/2 half
    G[sl(nf - h, nf - h + 1)] += 0.5 * F[sl(h, h + 1)]  # Nyquist, -nc/2 half
    return G


def spectral_interpolate(f, shape_c, shape_f):
    """Periodic band-limited interpolation of a field on the shape_c lattice (z-fastest site
    order) onto the finer shape_f lattice of the same box.  Exact for trigonometric polynomials
    of the coarse lattice; real input gives real output."""
    shape_c, shape_f = tuple(shape_c), tuple(shape_f)
    if any(b < a for a, b in zip(shape_c, shape_f)):
        raise ValueError("spectral_interpolate: the target lattice must not be coarser")
    f = np.asarray(f)
    F = np.fft.fftn(f.reshape(shape_c))
    for ax in range(3):
        F = _upsample_axis(F, shape_c[ax], shape_f[ax], ax)
    g = np.fft.ifftn(F) * (np.prod(shape_f) / np.prod(shape_c))
    g = g.reshape(-1)
    return g.real.copy() if np.isrealobj(f) else g


@dataclass
class Level:
    shape: tuple          # points per direction
    dx: float             # spacing in units of the finest lattice
    s: float              # dx^2: the factor from physical to scaled (unit-spacing) units
    g: float              # coupling in scaled units
    U0: float             # uniform Hartree shift in scaled units
    workload: object      # scaled problem: mu s, U = U0, Delta = s Delta0 x vortex ansatz
    phase: np.ndarray     # unit phase field of the ansatz, held fixed by the loop


def make_level(shape_f, ratio: float, mu: float, delta0: float, centers, charges, coupling) -> Level:
    """The scaled problem of the level with `ratio` times the finest lattice's points.
    centers: vortex positions in units of the finest spacing, measured from the box centre.
    coupling(nx, ny, nz, mu, delta0) -> (g, U0) solves a level's uniform gap equation."""
    import workloads as wk
    shape = level_shape(shape_f, ratio)
    dx = 1.0 / ratio
    s = dx * dx
    g, U0 = coupling(*shape, s * mu, s * delta0)
    D = wk.vortex_pairing(*shape, s * delta0, [(x * ratio, y * ratio) for x, y in centers], list(charges))
    w = wk.Workload(f"level_{shape[0]}x{shape[1]}x{shape[2]}", *shape, s * mu, np.full(int(np.prod(shape)), U0), D,
                    {"Delta0": s * delta0, "dx": dx})
    return Level(shape, dx, s, g, U0, w, np.exp(1j * np.angle(D)))


def multigrid_start(solve, coupling, mu: float, delta0: float, centers, charges, shape_f, ratios,
                    tol_coarse: float = 1e-4):
    """Start fields for the loop on the finest lattice.

    solve(workload, g, U, Delta, tol) -> (iterations, U, Delta) runs the loop on one level (in its
    scaled units, phase of workload.Delta held fixed); coupling as for make_level.  ratios: the
    coarser levels, e.g. (0.6, 0.8) for 60 and 80 points ahead of 100.  Each coarse level is
    converged to max|dn| <= tol_coarse per unit volume.
    Returns (U, Delta, iterations per coarse level) on the finest lattice in its own units."""
    ratios = sorted(float(r) for r in ratios)
    if any(not 0 < r < 1 for r in ratios):
        raise ValueError("multigrid_start: the coarse levels need ratios in (0, 1)")
    levels = [make_level(shape_f, r, mu, delta0, centers, charges, coupling) for r in ratios]
    fine = make_level(shape_f, 1.0, mu, delta0, centers, charges, coupling)
    its, prev = [], None
    for lv in levels + [fine]:
        U, D = lv.workload.U.copy(), lv.workload.Delta.copy()
        if prev is not None:
            pshape, dU, A = prev
            U = lv.U0 + lv.s * spectral_interpolate(dU, pshape, lv.shape)
            D = lv.s * spectral_interpolate(A, pshape, lv.shape) * lv.phase
        if lv is fine:
            return U, D, its
        it, Uc, Dc = solve(lv.workload, lv.g, U, D, tol_coarse * lv.dx ** 3)
        its.append(int(it))
        prev = (lv.shape, (np.asarray(Uc) - lv.U0) / lv.s, np.real(np.asarray(Dc) * np.conj(lv.phase)) / lv.s)


def main():
    """Plain start against the multigrid start on one seeded vortex state (GPU): the first seed,
    counting up from --seed, whose state has at least one vortex."""
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, default=16)
    ap.add_argument("--ratios", type=float, nargs="+", default=[0.5, 0.75])
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--tol-coarse", type=float, default=1e-4)
    a = ap.parse_args()
    import torch
    from . import Context, fno
    ctx = Context(0)
    seed = a.seed
    while not fno.sample(seed, a.grid).meta["centers"]:    # the first seeded state with a vortex
        seed += 1
    w = fno.sample(seed, a.grid)
    d0 = w.meta["Delta0"]
    centers = w.meta["centers"]
    charges = [1 if i % 2 == 0 else -1 for i in range(len(centers))]
    g, U0 = fno.coupling_for_gap(w.nx, w.ny, w.nz, w.mu, d0)

    def solve(wl, gl, U, D, tol):
        it, _, Uc, Dc, _ = fno.scf_solve(ctx, wl, gl, U, D, tol=tol)
        return it, Uc, Dc

    it0, t0, _, _, ok0 = fno.scf_solve(ctx, w, g, np.full(w.V, U0), w.Delta.copy(), tol=a.tol)
    torch.cuda.synchronize()
    t = time.perf_counter()
    U, D, its = multigrid_start(solve, fno.coupling_for_gap, w.mu, d0, centers, charges, (w.nx, w.ny, w.nz),
                                a.ratios, a.tol_coarse)
    t_coarse = time.perf_counter() - t
    it1, t1, _, _, ok1 = fno.scf_solve(ctx, w, g, U, D, tol=a.tol)
    print(json.dumps({"workload": f"{w.name}, {a.grid}^3 (N={w.N}), {len(centers)} vortices",
                      "levels": [list(level_shape((w.nx, w.ny, w.nz), r)) for r in sorted(a.ratios)],
                      "tol": a.tol, "plain": {"iterations": it0, "seconds": t0, "converged": ok0},
                      "multigrid": {"coarse_iterations": its, "coarse_seconds": t_coarse, "iterations": it1,
                                    "seconds": t1, "converged": ok1}}))


if __name__ == "__main__":
    main()
