"""The self-consistent step of a z-invariant state through its kz blocks.

When U(x, y) and Delta(x, y) do not depend on z (straight z-vortices, the learned-guess states of
the paper's training set), the quasiparticle wavefunctions of Eq. (stHpsi) on the nx x ny x nz grid
are phi(x, y) e^{i kz z} / sqrt(nz).  The BdG matrix then splits into nz blocks
H_kz = H_perp + (kz^2 / 2) tau_z of order 2 nx ny, one per kz = 2 pi m / nz (m = -nz/2 .. nz/2-1,
the z part of the spectral kinetic operator; tau_z = +1 on u, -1 on v, i.e. the block is the
nx x ny x 1 matrix at mu - kz^2/2).  The densities of Eq. (densities2) over the window
0 < E < Ec are the block densities averaged over kz,

    n(x, y) = (1/nz) sum_kz n_kz(x, y),     nu(x, y) = (1/nz) sum_kz nu_kz(x, y),

because |phi e^{i kz z} / sqrt(nz)|^2 = |phi|^2 / nz and the 3-D spectrum is the union of the
block spectra.  The blocks kz and -kz coincide (H depends on kz^2 only), so only m = 0 .. nz/2
is solved: m = 0 and the Nyquist block m = -nz/2 once, every other |m| twice.

The update is the one of bdg_scf_step (the stated contact functional): U_out = -g n / 2,
Delta_out = g nu (or g Re(nu e^{-i theta}) e^{i theta} with a fixed phase), mixed with weight
alpha.  A step on the nx x ny x nz grid costs about nz/2 + 1 solves of order 2 nx ny instead of one
of order 2 nx ny nz (for 24^3: 13 blocks of order 1152 against one of order 27648).

The block solver and the block densities are callables, so that the same reduction drives the
library (`library_solver`: bdg_build + bdg_heev_batched, and bdg_densities, all on the GPU) and,
in the tests, the oracle.
"""
from __future__ import annotations

import math


def kz_blocks(nz: int):
    """[(kz, multiplicity)] for kz = 2 pi m / nz, m = 0 .. nz/2.  nz is even or 1, as every grid
    dimension of the library (the even lattice's k set includes the Nyquist mode m = -nz/2)."""
    if nz < 1 or (nz > 1 and nz % 2):
        raise ValueError("kz_blocks: nz must be even or 1")
    out = []
    for m in range(0, nz // 2 + 1):
        if 2 * m == nz:
            mult = 1                       # the Nyquist block (m = -nz/2 only)
        elif m == 0:
            mult = 1
        else:
            mult = 2                       # m and -m
        out.append((2.0 * math.pi * m / nz, mult))
    assert sum(mu for _, mu in out) == nz
    return out


def kz_densities(nz: int, solve_all, densities):
    """(n, nu) of the z-invariant state averaged over its kz blocks.

    solve_all(kz_list) -> [(w, Z), ...] for the blocks at those kz;
    densities(w, Z) -> (n_kz, nu_kz) on the nx x ny grid (array-likes supporting + and *)."""
    blocks = kz_blocks(nz)
    sols = solve_all([k for k, _ in blocks])
    n = nu = None
    for (_, mult), (w, Z) in zip(blocks, sols):
        nk, nuk = densities(w, Z)
        n = mult * nk if n is None else n + mult * nk
        nu = mult * nuk if nu is None else nu + mult * nuk
    return n / nz, nu / nz


def scf_step_kz(nz: int, solve_all, densities, U, Delta, g: float, alpha: float = 0.3, phase=None):
    """One self-consistent step of a z-invariant state: blocks -> eigenpairs -> (n, nu) averaged
    over kz -> mixed update of (U, Delta).  Returns (U_new, Delta_new, n, nu)."""
    n, nu = kz_densities(nz, solve_all, densities)
    U_out = -g * n / 2.0
    if phase is None:
        D_out = g * nu
    else:
        D_out = g * (nu * phase.conj()).real * phase
    return (1.0 - alpha) * U + alpha * U_out, (1.0 - alpha) * Delta + alpha * D_out, n, nu


def library_solver(ctx, grid2d, mu: float, U2d, Delta2d, prec: str = "fp64", T: float = 0.0,
                   Ec: float = math.pi ** 2 / 2, ph: bool = True):
    """(solve_all, densities) for scf_step_kz on the GPU: the blocks by bdg_build at
    mu - kz^2/2 on the (nx, ny, 1) grid and one bdg_heev_batched call (particle-hole half solve
    per block with `ph`: every block is a BdG matrix); the block densities by bdg_densities.
    U2d and Delta2d are read when solve_all is called."""
    nx, ny = grid2d

    def solve_all(kz_list):
        mats = ctx.build_kz_blocks((nx, ny), mu, U2d, Delta2d, kz_list)
        return ctx.heev_batched(mats, prec, ph=ph, overwrite=True)

    def densities(w, Z):
        return ctx.densities((nx, ny, 1), w, Z, T=T, Ec=Ec)

    return solve_all, densities
