"""Time evolution of the quasiparticle wavefunctions (bdg_td_evolve, Eq. (TDSLDA)) against the
FP64 oracle (oracle/tdslda.py) on the same seeded initial states: the states and the densities
after several steps, element by element.  The step counts cross the switch from the RK4 start
to the Adams-Bashforth-Moulton steps.  The last case has the size of the single-vortex
workload (16^3 grid, N = 8192) with 512 evolved states."""
import numpy as np
import pytest

import oracle
import oracle.tdslda as td
import workloads as wk
from tests.gpu_common import ctx, torch

pytestmark = pytest.mark.gpu


def _random_states(N, nq, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((N, nq)) + 1j * rng.standard_normal((N, nq)))
    E0 = np.sort(rng.uniform(0.05, np.pi ** 2 / 2 - 0.05, nq))
    return Q, E0


def _window(w):
    ev, Z = oracle.heev(oracle.build(w))
    sel = np.nonzero((ev > 0) & (ev < np.pi ** 2 / 2))[0]
    return ev[sel], Z[:, sel]


def _run(w, g, E0, Psi0, dt, nsteps, T=0.0, U_ext=None, tol=1e-11):
    import paper_2310_03341_b300 as bdg
    grid = (w.nx, w.ny, w.nz)
    Psi_o, n_o, nu_o = td.evolve(grid, w.mu, g, Psi0, E0, dt, nsteps, T=T, U_ext=U_ext, threads=8)
    Pd = bdg.colmajor(torch.tensor(Psi0, dtype=torch.complex128, device="cuda"))
    Ed = torch.tensor(E0, dtype=torch.float64, device="cuda")
    Ud = torch.tensor(U_ext, dtype=torch.float64, device="cuda") if U_ext is not None else None
    n_g, nu_g = ctx().td_evolve(grid, Ed, Pd, dt, nsteps, w.mu, g, T=T, U_ext=Ud)
    torch.cuda.synchronize()
    scale = np.max(np.abs(Psi_o))
    assert np.max(np.abs(Pd.cpu().numpy() - Psi_o)) <= tol * scale
    assert np.max(np.abs(n_g.cpu().numpy() - n_o)) <= tol * np.max(np.abs(n_o))
    assert np.max(np.abs(nu_g.cpu().numpy() - nu_o)) <= tol * max(np.max(np.abs(nu_o)), 1e-300)
    return Psi_o


def test_td_vortex_window_states_match_the_oracle():
    w = wk.random_small(4, 4, 4, seed=2, n_vortices=1)
    g, _ = oracle.gap_coupling(w.nx, w.ny, w.nz, w.mu, 0.3)
    E0, Psi0 = _window(w)
    Psi = _run(w, g, E0, Psi0, 0.02, 12, U_ext=w.U)
    assert np.max(np.abs(Psi - Psi0)) > 1e-3          # the states really moved


def test_td_ragged_grid_finite_temperature_matches_the_oracle():
    w = wk.random_small(6, 4, 10, seed=4, n_vortices=2)
    g, _ = oracle.gap_coupling(w.nx, w.ny, w.nz, w.mu, 0.3)
    E0, Psi0 = _window(w)
    _run(w, g, E0, Psi0, 0.015, 7, T=0.05)


def test_td_zero_steps_returns_the_initial_state_and_its_densities():
    w = wk.random_small(4, 4, 2, seed=5, n_vortices=1)
    E0, Psi0 = _window(w)
    _run(w, 1.0, E0, Psi0, 0.01, 0, tol=1e-13)


def test_td_single_vortex_size_matches_the_oracle():
    w = wk.c2_single_vortex()
    g, _ = oracle.gap_coupling(w.nx, w.ny, w.nz, w.mu, 0.3)
    Psi0, E0 = _random_states(w.N, 512, seed=21)
    _run(w, g, E0, Psi0, 0.01, 6, U_ext=w.U)
