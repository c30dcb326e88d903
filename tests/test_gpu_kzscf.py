"""The kz-block reduction of the self-consistent step on the GPU (paper_2310_03341_b300.kzscf with
the library's bdg_build / bdg_heev_batched / bdg_densities per block) against the FP64 oracle's
full nx x ny x nz problem: densities and one mixed update of a z-invariant vortex state."""
import math

import numpy as np
import pytest

import oracle
import workloads as wk
from paper_2310_03341_b300 import kzscf
from tests.gpu_common import ctx, torch

pytestmark = pytest.mark.gpu


def _state(nx, ny, nz, seed):
    D2 = wk.vortex_pairing(nx, ny, 1, 0.35, [(0.3, -0.2)], [1])
    U2 = -0.3 + wk.smooth_field((nx, ny), 2.0, seed, 0.08)
    w3 = wk.Workload("z_invariant", nx, ny, nz, 0.5, np.repeat(U2, nz), np.repeat(D2, nz))
    return w3, U2, D2


@pytest.mark.parametrize("nx,ny,nz,prec", [(4, 4, 6, "fp64"), (6, 4, 8, "fp64"), (4, 4, 6, "fp32")])
def test_kz_block_densities_match_the_3d_oracle(nx, ny, nz, prec):
    w3, U2, D2 = _state(nx, ny, nz, seed=3)
    ev, Z = oracle.heev(oracle.build(w3), vectors=True)
    n3, nu3 = oracle.densities(ev, Z, w3.V, 0.0, math.pi ** 2 / 2)
    c = ctx()
    U = torch.tensor(U2, dtype=torch.float64, device="cuda")
    D = torch.tensor(D2, dtype=torch.complex128, device="cuda")
    solve_all, dens = kzscf.library_solver(c, (nx, ny), w3.mu, U, D, prec=prec)
    n2, nu2 = kzscf.kz_densities(nz, solve_all, dens)
    tol = 1e-11 if prec == "fp64" else 1e-5
    n2 = np.repeat(n2.cpu().numpy(), nz)
    nu2 = np.repeat(nu2.cpu().numpy(), nz)
    assert np.max(np.abs(n2 - n3)) <= tol * np.max(np.abs(n3))
    assert np.max(np.abs(nu2 - nu3)) <= tol * np.max(np.abs(nu3))


def test_kz_scf_step_matches_the_3d_oracle_step():
    nx, ny, nz = 4, 4, 6
    w3, U2, D2 = _state(nx, ny, nz, seed=5)
    g = 3.0
    U3n, D3n, _, _ = oracle.scf_step(w3, g, alpha=0.3)
    c = ctx()
    U = torch.tensor(U2, dtype=torch.float64, device="cuda")
    D = torch.tensor(D2, dtype=torch.complex128, device="cuda")
    solve_all, dens = kzscf.library_solver(c, (nx, ny), w3.mu, U, D, prec="fp64")
    Un, Dn, _, _ = kzscf.scf_step_kz(nz, solve_all, dens, U, D, g, alpha=0.3)
    assert np.max(np.abs(np.repeat(Un.cpu().numpy(), nz) - U3n)) <= 1e-11 * np.max(np.abs(U3n))
    assert np.max(np.abs(np.repeat(Dn.cpu().numpy(), nz) - D3n)) <= 1e-11 * np.max(np.abs(D3n))
