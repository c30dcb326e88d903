"""The kz-block reduction of the self-consistent step (paper_2310_03341_b300.kzscf), on the CPU with
the FP64 oracle as the block solver: for a z-invariant state the block densities averaged over kz
equal the densities of the full nx x ny x nz problem at every site, and so does the mixed update of
one SCF step; the block list covers every kz of the lattice once."""
import math

import numpy as np
import pytest

import oracle
import workloads as wk
from paper_2310_03341_b300 import kzscf


def z_invariant(nx, ny, nz, seed, mu=0.5, d0=0.35):
    """A straight z-vortex and a seeded 2-D U: the 3-D workload and its (nx, ny, 1) fields."""
    D2 = wk.vortex_pairing(nx, ny, 1, d0, [(0.3, -0.2)], [1])
    U2 = -0.3 + wk.smooth_field((nx, ny), 2.0, seed, 0.08)
    U3 = np.repeat(U2, nz)                      # z-fastest site order
    D3 = np.repeat(D2, nz)
    w3 = wk.Workload("z_invariant", nx, ny, nz, mu, U3, D3)
    return w3, U2, D2


def oracle_solver(nx, ny, mu, U2, D2, T=0.0, Ec=math.pi ** 2 / 2):
    def solve_all(kz_list):
        out = []
        for k in kz_list:
            wb = wk.Workload("block", nx, ny, 1, mu - 0.5 * k * k, U2, D2)
            out.append(oracle.heev(oracle.build(wb), vectors=True))
        return out

    def densities(w, Z):
        return oracle.densities(w, Z, nx * ny, T, Ec)

    return solve_all, densities


@pytest.mark.parametrize("nz", [1, 2, 6, 8])
def test_kz_blocks_cover_the_lattice_once(nz):
    blocks = kzscf.kz_blocks(nz)
    full = sorted(round(abs(2 * math.pi * m / nz), 12) for m in range(-(nz // 2), nz - nz // 2))
    listed = sorted(round(k, 12) for k, mult in blocks for _ in range(mult))
    assert listed == full


@pytest.mark.parametrize("nx,ny,nz,T", [(4, 4, 6, 0.0), (4, 6, 8, 0.0), (4, 4, 4, 0.05), (6, 4, 1, 0.0)])
def test_block_densities_equal_the_3d_densities(nx, ny, nz, T):
    w3, U2, D2 = z_invariant(nx, ny, nz, seed=3)
    ev, Z = oracle.heev(oracle.build(w3), vectors=True)
    n3, nu3 = oracle.densities(ev, Z, w3.V, T, math.pi ** 2 / 2)
    solve_all, dens = oracle_solver(nx, ny, w3.mu, U2, D2, T)
    n2, nu2 = kzscf.kz_densities(nz, solve_all, dens)
    scale = max(np.max(np.abs(n3)), 1e-300)
    assert np.max(np.abs(np.repeat(n2, nz) - n3)) <= 1e-12 * scale
    assert np.max(np.abs(np.repeat(nu2, nz) - nu3)) <= 1e-12 * max(np.max(np.abs(nu3)), 1e-300)


def test_scf_step_equals_the_3d_step():
    nx, ny, nz = 4, 4, 6
    w3, U2, D2 = z_invariant(nx, ny, nz, seed=5)
    g = 3.0
    U3n, D3n, n3, nu3 = oracle.scf_step(w3, g, alpha=0.3)
    solve_all, dens = oracle_solver(nx, ny, w3.mu, U2, D2)
    U2n, D2n, n2, nu2 = kzscf.scf_step_kz(nz, solve_all, dens, U2, D2, g, alpha=0.3)
    assert np.max(np.abs(np.repeat(U2n, nz) - U3n)) <= 1e-12 * np.max(np.abs(U3n))
    assert np.max(np.abs(np.repeat(D2n, nz) - D3n)) <= 1e-12 * np.max(np.abs(D3n))


def test_odd_nz_is_rejected():
    with pytest.raises(ValueError):
        kzscf.kz_blocks(5)


def test_a_dropped_multiplicity_is_caught():
    """Planted mistake: counting each +-kz pair once breaks the equality."""
    nx, ny, nz = 4, 4, 6
    w3, U2, D2 = z_invariant(nx, ny, nz, seed=3)
    ev, Z = oracle.heev(oracle.build(w3), vectors=True)
    n3, _ = oracle.densities(ev, Z, w3.V, 0.0, math.pi ** 2 / 2)
    solve_all, dens = oracle_solver(nx, ny, w3.mu, U2, D2)
    blocks = kzscf.kz_blocks(nz)
    sols = solve_all([k for k, _ in blocks])
    n_once = sum(dens(w, Z)[0] for w, Z in sols) / nz
    assert np.max(np.abs(np.repeat(n_once, nz) - n3)) > 1e-3 * np.max(np.abs(n3))


def test_fno_kz_loop_matches_the_3d_oracle_loop():
    """fno.scf_solve_kz (the learned-guess driver's kz path) with the oracle as block solver, three
    fixed-phase steps, against three oracle.scf_step calls on the full grid."""
    torch = pytest.importorskip("torch")
    from paper_2310_03341_b300 import fno
    nx, ny, nz = 4, 4, 4
    w3, U2, D2 = z_invariant(nx, ny, nz, seed=7)
    g, alpha = 3.0, 0.7
    phase = fno.fixed_phase(w3)

    def solver(U2t, D2t):
        def solve_all(kz_list):
            Uc, Dc = U2t.numpy(), D2t.numpy()
            return [oracle.heev(oracle.build(wk.Workload("b", nx, ny, 1, w3.mu - 0.5 * k * k, Uc, Dc)),
                                vectors=True) for k in kz_list]

        def dens(w, Z):
            n, nu = oracle.densities(w, Z, nx * ny, 0.0, math.pi ** 2 / 2)
            return torch.tensor(n), torch.tensor(nu)
        return solve_all, dens

    it, _, Uk, Dk, _ = fno.scf_solve_kz(None, w3, g, w3.U, w3.Delta, tol=0.0, max_iter=3, alpha=alpha,
                                        device="cpu", solver=solver)
    assert it == 3
    wr = wk.Workload("r", nx, ny, nz, w3.mu, w3.U.copy(), w3.Delta.copy())
    for _ in range(3):
        wr.U, wr.Delta, _, _ = oracle.scf_step(wr, g, alpha=alpha, phase=phase)
    assert np.max(np.abs(Uk - wr.U)) <= 1e-11 * np.max(np.abs(wr.U))
    assert np.max(np.abs(Dk - wr.Delta)) <= 1e-11 * np.max(np.abs(wr.Delta))


def test_fno_kz_loop_rejects_z_dependent_fields():
    pytest.importorskip("torch")
    from paper_2310_03341_b300 import fno
    w3, _, _ = z_invariant(4, 4, 4, seed=7)
    U = w3.U.copy()
    U[1] += 0.1
    with pytest.raises(ValueError):
        fno.scf_solve_kz(None, w3, 3.0, U, w3.Delta, device="cpu", solver=lambda a, b: (None, None))


def _oracle_kz_solver(torch, w3):
    nx, ny = w3.nx, w3.ny

    def solver(U2t, D2t):
        def solve_all(kz_list):
            Uc, Dc = U2t.numpy(), D2t.numpy()
            return [oracle.heev(oracle.build(wk.Workload("b", nx, ny, 1, w3.mu - 0.5 * k * k, Uc, Dc)),
                                vectors=True) for k in kz_list]

        def dens(w, Z):
            n, nu = oracle.densities(w, Z, nx * ny, 0.0, math.pi ** 2 / 2)
            return torch.tensor(n), torch.tensor(nu)
        return solve_all, dens
    return solver


def test_fno_kz_loop_resumes_from_its_checkpoint(tmp_path):
    """Two steps, then a resumed call to four, equal four straight steps; a converged checkpoint
    returns at once; the checkpoint holds the fields on the full grid."""
    torch = pytest.importorskip("torch")
    from paper_2310_03341_b300 import fno, scf_state
    w3, _, _ = z_invariant(4, 4, 4, seed=7)
    g, alpha = 3.0, 0.7
    solver = _oracle_kz_solver(torch, w3)
    ck = str(tmp_path / "kz.npz")
    it2, *_ = fno.scf_solve_kz(None, w3, g, w3.U, w3.Delta, tol=0.0, max_iter=2, alpha=alpha, checkpoint=ck,
                               device="cpu", solver=solver)
    assert it2 == 2 and scf_state.load(ck)["U"].shape == (w3.V,)
    it4, _, Ur, Dr, _ = fno.scf_solve_kz(None, w3, g, w3.U, w3.Delta, tol=0.0, max_iter=4, alpha=alpha,
                                         checkpoint=ck, device="cpu", solver=solver)
    _, _, Us, Ds, _ = fno.scf_solve_kz(None, w3, g, w3.U, w3.Delta, tol=0.0, max_iter=4, alpha=alpha,
                                       device="cpu", solver=solver)
    assert it4 == 4
    assert np.array_equal(Ur, Us) and np.array_equal(Dr, Ds)
    st = scf_state.load(ck)
    assert st["iteration"] == 4 and len(st["dn_history"]) == 4
    # a loose tolerance marks the stored state converged: the next call does no step
    it_done, *_ = fno.scf_solve_kz(None, w3, g, w3.U, w3.Delta, tol=1e9, max_iter=10, alpha=alpha,
                                   checkpoint=ck, device="cpu", solver=solver)
    assert it_done == 4
