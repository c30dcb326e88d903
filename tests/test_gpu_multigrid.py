"""Multigrid start of the self-consistent loop on the GPU (paper, "Performance of the Matrix
Diagonalization Algorithm": the solution converged on a coarser lattice of the same box starts the
loop on the finer one).  Every level's loop is bdg_scf_step (FP64 eigensolve, the stated contact
functional, fixed vortex phase).  The case is the one of the CPU test: one vortex in an 8x8x4 box,
coarse level 4x4x2.  Checked: the plain-start loop follows the oracle's loop step for step (same
iteration count, same converged fields), and the multigrid start converges in clearly fewer fine
iterations to the same solution."""
import numpy as np
import pytest

import oracle
import paper_2310_03341_b300.multigrid as mg
import workloads as wk
from paper_2310_03341_b300 import fno
from tests.gpu_common import ctx

pytestmark = pytest.mark.gpu


def _oracle_loop(w, g, U, D, tol, alpha=0.7, max_iter=300):
    ph = np.exp(1j * np.angle(w.Delta))
    wl = wk.Workload("loop", w.nx, w.ny, w.nz, w.mu, np.array(U, dtype=float), np.array(D, dtype=complex), {})
    n_prev = np.zeros(w.V)
    for it in range(1, max_iter + 1):
        wl.U, wl.Delta, n, _ = oracle.scf_step(wl, g, alpha=alpha, phase=ph, threads=8)
        dn = np.max(np.abs(n - n_prev))
        n_prev = n
        if it > 1 and dn <= tol:
            return it, wl.U, wl.Delta
    return max_iter, wl.U, wl.Delta


def test_multigrid_start_on_the_gpu():
    c = ctx()
    mu, d0, centers, charges = 0.5, 0.45, [(0.3, 0.2)], [1]
    shape, tol = (8, 8, 4), 1e-5
    fine = mg.make_level(shape, 1.0, mu, d0, centers, charges, fno.coupling_for_gap)

    def solve(wl, g, U, D, tl):
        it, _, Uc, Dc, ok = fno.scf_solve(c, wl, g, U, D, tol=tl, max_iter=300, alpha=0.7, prec="fp64")
        assert ok
        return it, Uc, Dc

    it_plain, Up, Dp = solve(fine.workload, fine.g, fine.workload.U, fine.workload.Delta, tol)
    it_o, Uo, Do = _oracle_loop(fine.workload, fine.g, fine.workload.U, fine.workload.Delta, tol)
    assert abs(it_plain - it_o) <= 1
    assert np.max(np.abs(Up - Uo)) < 1e-7 and np.max(np.abs(Dp - Do)) < 1e-6
    U, D, its = mg.multigrid_start(solve, fno.coupling_for_gap, mu, d0, centers, charges, shape, [0.5])
    assert len(its) == 1 and its[0] > 1
    it_mg, Um, Dm = solve(fine.workload, fine.g, U, D, tol)
    assert it_mg < 0.6 * it_plain
    assert np.max(np.abs(Um - Up)) < 2e-3 and np.max(np.abs(Dm - Dp)) < 2e-2
