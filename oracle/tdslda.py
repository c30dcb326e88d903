"""FP64 CPU oracle for the time evolution of the quasiparticle wavefunctions --
TEST INFRASTRUCTURE ONLY (same rules as the rest of ``oracle``: only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may import it; the CUDA
library shares no code with it).

What it computes.  Every quasiparticle wavefunction phi_n = (u_n, v_n) of the
window evolves under the same quasiparticle Hamiltonian (paper, Eq. (TDSLDA)):

    i d phi_n / dt = H(t) phi_n,   H = [[h, Delta], [Delta^*, -h^*]],
    h = T + U(r, t) - mu,

with T the spectral kinetic operator of the static problem (Eq. (stHpsi)) and
(U, Delta) given at every instant by the local densities of the evolved
states (Eq. (densities2) with the occupation of each state fixed at its
initial value: f_T(E_n) on |u_n|^2, f_T(-E_n) on |v_n|^2).  The functional is
the stated contact substitute of the static loop, with an optional static
external potential:  U = U_ext - g n / 2,  Delta = g nu.

Time stepping (paper, "Performance of the Time Evolution Algorithm"): the
fifth-order Adams-Bashforth-Moulton predictor-corrector, with H (that is,
the densities, U and Delta) evaluated twice per step -- at the predicted
state and at the corrected one (predict, evaluate, correct, evaluate):

    predictor  P = phi_n + dt sum_k b_k F_{n-k},   b = (1901, -2774, 2616, -1274, 251) / 720,
    corrector  phi_{n+1} = phi_n + dt (a_0 F(P) + sum_{k>=1} a_k F_{n+1-k}),
                                              a = (251, 646, -264, 106, -19) / 720,
    F(phi) = -i H[phi] phi.

Reading (the paper does not say how the multistep history is started): the
first four steps are classical fourth-order Runge-Kutta steps, so that
F_0 .. F_4 exist when the first ABM step is taken.
"""
from __future__ import annotations

import numpy as np

from . import apply, fermi

AB5 = np.array([1901.0, -2774.0, 2616.0, -1274.0, 251.0]) / 720.0   # F_n, F_{n-1}, ..., F_{n-4}
AM5 = np.array([251.0, 646.0, -264.0, 106.0, -19.0]) / 720.0        # F(P), F_n, F_{n-1}, F_{n-2}, F_{n-3}


class _Fields:
    """The minimal workload record that ``oracle.apply`` reads."""

    def __init__(self, nx, ny, nz, mu, U, Delta):
        self.nx, self.ny, self.nz, self.mu, self.U, self.Delta = nx, ny, nz, mu, U, Delta


def weights(E0: np.ndarray, T: float):
    """Occupation weights (f_T(E_n), f_T(-E_n)) of the evolved states, fixed in time."""
    return fermi(E0, T), fermi(-np.asarray(E0, dtype=np.float64), T)


def densities(Psi: np.ndarray, V: int, fp: np.ndarray, fm: np.ndarray):
    """n = 2 sum (|v|^2 f(-E) + |u|^2 f(E)),  nu = sum u v^* (f(-E) - f(E))  (Eq. (densities2))."""
    u, v = Psi[:V], Psi[V:]
    n = 2.0 * ((np.abs(v) ** 2) @ fm + (np.abs(u) ** 2) @ fp)
    nu = (u * np.conj(v)) @ (fm - fp)
    return n, nu


def fields(n: np.ndarray, nu: np.ndarray, g: float, U_ext):
    """The contact functional: U = U_ext - g n / 2, Delta = g nu."""
    U = -0.5 * g * n
    if U_ext is not None:
        U = U + U_ext
    return U, g * nu


def rhs(grid, mu, g, U_ext, fp, fm, Psi, threads=0):
    """F(Psi) = -i H[Psi] Psi with H built from the densities of Psi."""
    nx, ny, nz = grid
    V = nx * ny * nz
    n, nu = densities(Psi, V, fp, fm)
    U, D = fields(n, nu, g, U_ext)
    return -1j * apply(_Fields(nx, ny, nz, mu, U, D), Psi, threads)


def evolve(grid, mu: float, g: float, Psi0: np.ndarray, E0: np.ndarray, dt: float, nsteps: int, T: float = 0.0,
           U_ext=None, threads: int = 0):
    """Psi(t = nsteps dt) from Psi(0) (2V x nq, columns the evolved states, energies E0 for the
    occupation weights).  Returns (Psi, n, nu) at the final time."""
    nx, ny, nz = grid
    V = nx * ny * nz
    fp, fm = weights(E0, T)
    F = lambda X: rhs(grid, mu, g, U_ext, fp, fm, X, threads)   # noqa: E731
    Psi = np.array(Psi0, dtype=np.complex128, order="F")
    hist = [F(Psi)]                   # F_0
    for step in range(nsteps):
        if len(hist) < 5:
            # classical RK4 while the multistep history is being built
            k1 = hist[-1]
            k2 = F(Psi + 0.5 * dt * k1)
            k3 = F(Psi + 0.5 * dt * k2)
            k4 = F(Psi + dt * k3)
            Psi = Psi + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        else:
            P = Psi + dt * sum(AB5[k] * hist[-1 - k] for k in range(5))
            FP = F(P)
            Psi = Psi + dt * (AM5[0] * FP + sum(AM5[k] * hist[-k] for k in range(1, 5)))
        hist.append(F(Psi))
        if len(hist) > 5:
            hist.pop(0)
    n, nu = densities(Psi, V, fp, fm)
    return Psi, n, nu
