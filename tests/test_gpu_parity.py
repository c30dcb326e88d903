"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (relative to the spectral radius rho = max |lambda|):
  FP64 path        eigenvalues <= 1e-12, residual ||Hz - lambda z|| <= 1e-12,
                   orthogonality <= 1e-10;
  FP32 / BF16x3    eigenvalues <= 1e-5, residual <= 1e-4 (FP32 unit round-off
                   6e-8, or 2^-17 for split bf16 products, times the growth of
                   a two-stage reduction);
  reduced + refine eigenvalues <= 1e-12, residual <= 1e-11 -- the 1e-10 target
                   with margin.
Eigenvectors are compared through what is unique: eigenvalues, residuals,
orthogonality and, for isolated eigenvalues, |<z_gpu, z_oracle>| = 1
(degenerate eigenspaces admit any orthonormal basis).
"""
import numpy as np
import pytest

import oracle
import workloads as wk
from tests import pins
from tests.gpu_common import ctx, dev_fields, gpu_eig, isolated, torch

pytestmark = pytest.mark.gpu

# sizes span several band panels (b = 32 in FP64, 64 in FP32) and ragged tails
SHAPES = [(2, 2, 4), (4, 4, 6), (6, 6, 6), (4, 6, 10), (8, 8, 8)]


def _case(shape, seed=1):
    if shape == (8, 8, 8):
        return wk.c1_uniform()
    return wk.random_small(*shape, seed=seed, n_vortices=2)


@pytest.mark.parametrize("shape", [(2, 2, 4), (4, 4, 6), (6, 8, 4), (8, 8, 8)])
def test_build_matches_oracle(shape):
    w = _case(shape)
    U, D = dev_fields(w)
    H = ctx().build((w.nx, w.ny, w.nz), w.mu, U, D).cpu().numpy()
    Ho = oracle.build(w)
    assert np.max(np.abs(H - Ho)) < 1e-14 * max(1.0, np.max(np.abs(Ho)))


@pytest.mark.parametrize("shape", SHAPES)
def test_heev_fp64_matches_oracle(shape):
    w = _case(shape)
    Ho = oracle.build(w)
    ew, Zo = oracle.heev(Ho)
    ev, Z, _ = gpu_eig(w, "fp64")
    rho = np.max(np.abs(ew))
    assert np.max(np.abs(ev - ew)) / rho <= 1e-12
    res = oracle.residuals(w, ev, Z)
    assert np.max(res) / rho <= 1e-12
    assert oracle.orthogonality(Z) <= 1e-10
    iso = isolated(ew)
    ov = np.abs(np.sum(Z[:, iso].conj() * Zo[:, iso], axis=0))
    assert np.min(ov) >= 1 - 1e-9


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "bf16x6", "bf16x9"])
@pytest.mark.parametrize("shape", SHAPES)
def test_heev_reduced_precision_matches_oracle(shape, prec):
    w = _case(shape)
    ew = oracle.heev(oracle.build(w), vectors=False)
    ev, Z, _ = gpu_eig(w, prec)
    rho = np.max(np.abs(ew))
    assert np.max(np.abs(ev - ew)) / rho <= 1e-5
    assert np.max(oracle.residuals(w, ev, Z)) / rho <= 1e-4
    assert oracle.orthogonality(Z) <= 1e-4


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "bf16x6", "bf16x9"])
@pytest.mark.parametrize("shape", SHAPES)
def test_refined_reduced_precision_reaches_fp64_accuracy(shape, prec):
    w = _case(shape)
    ew = oracle.heev(oracle.build(w), vectors=False)
    ev, Z, info = gpu_eig(w, prec, refine=5, tol=1e-13)
    rho = np.max(np.abs(ew))
    assert np.max(np.abs(ev - ew)) / rho <= 1e-12
    assert np.max(oracle.residuals(w, ev, Z)) / rho <= 1e-11
    assert oracle.orthogonality(Z) <= 1e-9
    resid, orth, iters, ok = info
    assert resid <= 1e-11 and iters >= 1


def _partner(Z):
    """Columns h-1-j of the particle-hole partners of columns h+j: (conj v, -conj u)."""
    n = Z.shape[0]
    h = n // 2
    up = Z[:, h:]
    P = np.concatenate([np.conj(up[h:]), -np.conj(up[:h])])
    return P[:, ::-1]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x9"])
@pytest.mark.parametrize("shape", SHAPES)
def test_heev_particle_hole_half_solve_matches_oracle(shape, prec):
    """BDG_HEEV_PH: only the upper half is solved, the lower half is the
    partner map; the result must match the oracle like the full solve."""
    w = _case(shape)
    ew = oracle.heev(oracle.build(w), vectors=False)
    ev, Z, _ = gpu_eig(w, prec, ph=True)
    assert ctx().last_modes()[0], "the half solve did not run"
    rho = np.max(np.abs(ew))
    fp64 = prec == "fp64"
    assert np.max(np.abs(ev - ew)) / rho <= (1e-12 if fp64 else 1e-5)
    assert np.max(oracle.residuals(w, ev, Z)) / rho <= (1e-12 if fp64 else 1e-4)
    assert oracle.orthogonality(Z) <= (1e-10 if fp64 else 1e-4)
    h = w.N // 2
    assert np.array_equal(ev[:h], -ev[h:][::-1])
    assert np.array_equal(Z[:, :h], _partner(Z))


@pytest.mark.parametrize("shape", [(4, 4, 6), (4, 6, 10), (8, 8, 8)])
def test_refine_particle_hole_reduction_matches_full_refinement(shape, monkeypatch):
    """The particle-hole refinement (G++, S++, K, L on half the columns) and
    the full one reach the same FP64-level pairs."""
    w = _case(shape)
    ew = oracle.heev(oracle.build(w), vectors=False)
    rho = np.max(np.abs(ew))
    for full in (False, True):
        if full:
            monkeypatch.setenv("BDG_REFINE_FULL", "1")
        else:
            monkeypatch.delenv("BDG_REFINE_FULL", raising=False)
        ev, Z, info = gpu_eig(w, "bf16x9", refine=6, tol=1e-12, ph=True)
        assert ctx().last_modes()[1] == (not full)
        assert np.max(np.abs(ev - ew)) / rho <= 1e-12
        assert np.max(oracle.residuals(w, ev, Z)) / rho <= 1e-11
        assert oracle.orthogonality(Z) <= 1e-9
        assert info[3]


def test_uniform_closed_form_on_gpu():
    """Config C1 against the closed form E_k = +-sqrt((k^2/2 - mu)^2 + Delta^2)."""
    w = wk.c1_uniform()
    ev, Z, _ = gpu_eig(w, "fp64")
    ref = pins.uniform_spectrum(8, 8, 8, 0.5, 0.0, 0.2)
    assert np.max(np.abs(ev - ref)) / np.max(np.abs(ref)) <= 1e-13


def test_particle_hole_pairing_on_gpu():
    w = wk.random_small(4, 6, 4, seed=4, n_vortices=2)
    ev, Z, _ = gpu_eig(w, "fp64")
    rho = np.max(np.abs(ev))
    assert np.max(np.abs(ev + ev[::-1])) / rho < 1e-13
    assert abs(np.sum(ev)) / rho < 1e-11
    f2 = pins.frobenius2_closed_form(w)
    assert abs(np.sum(ev ** 2) - f2) / f2 < 1e-12


@pytest.mark.parametrize("kind", ["diagonal", "zero", "tiny"])
def test_heev_degenerate_inputs(kind):
    c = ctx()
    if kind == "tiny":
        n = 2
        A = torch.tensor([[1.0, 2 - 1j], [2 + 1j, -3.0]], dtype=torch.complex128, device="cuda")
    else:
        n = 70
        d = torch.linspace(-2, 3, n, dtype=torch.float64)
        A = torch.diag(d).to(torch.complex128).cuda() if kind == "diagonal" else \
            torch.zeros(n, n, dtype=torch.complex128, device="cuda")
    An = A.cpu().numpy()
    for prec in ("fp64", "fp32"):
        ev, Z = c.heev(A, prec)
        ev, Z = ev.cpu().numpy(), Z.cpu().numpy()
        ref = np.linalg.eigvalsh(An)
        tol = 1e-13 if prec == "fp64" else 1e-6
        assert np.max(np.abs(ev - ref)) <= tol * max(1.0, np.max(np.abs(ref)))
        assert np.max(np.abs(An @ Z - Z * ev)) <= tol * max(1.0, np.max(np.abs(ref)))
        assert np.max(np.abs(Z.conj().T @ Z - np.eye(n))) <= (1e-12 if prec == "fp64" else 1e-5)


def test_heev_large_tight_cluster():
    """A cluster of 300 eigenvalues within 1e-9 of each other inside one unreduced tridiagonal
    block: the inverse-iteration path that takes a cluster per CTA, with Gram-Schmidt in chunks
    of 256 earlier members.  Eigenvalues against numpy, residuals and orthogonality."""
    rng = np.random.default_rng(11)
    n, k = 600, 300
    lam = np.concatenate([np.linspace(-3.0, -0.5, (n - k) // 2), 1.0 + 1e-9 * rng.random(k),
                          np.linspace(1.5, 4.0, n - k - (n - k) // 2)])
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    An = (Q * lam) @ Q.conj().T
    An = 0.5 * (An + An.conj().T)
    A = torch.tensor(An, dtype=torch.complex128, device="cuda")
    ev, Z = ctx().heev(A, "fp64")
    ev, Z = ev.cpu().numpy(), Z.cpu().numpy()
    ref = np.linalg.eigvalsh(An)
    assert np.max(np.abs(ev - ref)) <= 1e-13 * 4.0
    assert np.max(np.abs(An @ Z - Z * ev)) <= 1e-12 * 4.0
    assert np.max(np.abs(Z.conj().T @ Z - np.eye(n))) <= 1e-11


def test_heev_one_by_one():
    A = torch.tensor([[2.5]], dtype=torch.complex128, device="cuda")
    ev, Z = ctx().heev(A, "fp64")
    assert float(ev[0]) == 2.5 and abs(complex(Z[0, 0].item())) == 1.0


def test_invalid_arguments_are_rejected():
    import paper_2310_03341_b300 as bdg
    c = ctx()
    U = torch.zeros(3 * 4 * 4, dtype=torch.float64, device="cuda")
    D = torch.zeros(3 * 4 * 4, dtype=torch.complex128, device="cuda")
    with pytest.raises(bdg.BdgError) as e:
        c.build((3, 4, 4), 0.5, U, D)   # odd grid
    assert e.value.code == -1


@pytest.mark.parametrize("T", [0.0, 0.05])
@pytest.mark.parametrize("shape", [(4, 4, 6), (6, 4, 4)])
def test_densities_match_oracle(shape, T):
    w = wk.random_small(*shape, seed=3, n_vortices=1)
    ew, Zo = oracle.heev(oracle.build(w))
    n_o, nu_o = oracle.densities(ew, Zo, w.V, T=T)
    ev, Z, _ = gpu_eig(w, "fp64")
    evt = torch.tensor(ev, device="cuda")
    Zt = torch.tensor(Z, device="cuda")
    import paper_2310_03341_b300 as bdg
    nd, nu = ctx().densities((w.nx, w.ny, w.nz), evt, bdg.colmajor(Zt), T=T)
    assert np.max(np.abs(nd.cpu().numpy() - n_o)) < 1e-11
    assert np.max(np.abs(nu.cpu().numpy() - nu_o)) < 1e-11


def test_uniform_densities_closed_form_on_gpu():
    nx, ny, nz, mu, D0 = 4, 4, 6, 0.5, 0.2
    w = wk.uniform(nx, ny, nz, mu, 0.0, D0)
    ev, Z, _ = gpu_eig(w, "fp64")
    import paper_2310_03341_b300 as bdg
    nd, nu = ctx().densities((nx, ny, nz), torch.tensor(ev, device="cuda"),
                             bdg.colmajor(torch.tensor(Z, device="cuda")))
    xi = pins.lattice_k2half(nx, ny, nz) - mu
    E = np.sqrt(xi ** 2 + D0 ** 2)
    sel = E < np.pi ** 2 / 2
    n0 = 2.0 / w.V * np.sum(0.5 * (1 - xi[sel] / E[sel]))
    nu0 = 1.0 / w.V * np.sum(D0 / (2 * E[sel]))
    assert np.max(np.abs(nd.cpu().numpy() - n0)) < 1e-12
    assert np.max(np.abs(nu.cpu().numpy() - nu0)) < 1e-12


def test_scf_uniform_fixed_point_on_gpu():
    nx, ny, nz, mu, D0 = 4, 4, 4, 0.5, 0.25
    g, U0 = oracle.gap_coupling(nx, ny, nz, mu, D0)
    V = nx * ny * nz
    U = torch.full((V,), U0, dtype=torch.float64, device="cuda")
    D = torch.full((V,), D0, dtype=torch.complex128, device="cuda")
    n0, _, _ = oracle.uniform_sums(nx, ny, nz, mu, U0, D0)
    n_prev = torch.full((V,), n0, dtype=torch.float64, device="cuda")
    dn = ctx().scf_step((nx, ny, nz), U, D, n_prev, mu, g, alpha=1.0, prec="fp64")
    assert np.max(np.abs(U.cpu().numpy() - U0)) < 1e-11
    assert np.max(np.abs(D.cpu().numpy() - D0)) < 1e-11
    assert dn < 1e-11


@pytest.mark.parametrize("fixed_phase", [False, True])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_scf_step_matches_oracle(fixed_phase, prec):
    w = wk.random_small(4, 4, 6, seed=8, n_vortices=1, amplitude=0.3)
    g, _ = oracle.gap_coupling(w.nx, w.ny, w.nz, w.mu, 0.3)
    phase = np.exp(1j * np.angle(w.Delta)) if fixed_phase else None
    U1, D1, n1, _ = oracle.scf_step(w, g, alpha=0.3, phase=phase)
    U, D = dev_fields(w)
    n_prev = torch.zeros(w.V, dtype=torch.float64, device="cuda")
    ph = torch.tensor(phase, device="cuda") if fixed_phase else None
    dn = ctx().scf_step((w.nx, w.ny, w.nz), U, D, n_prev, w.mu, g, alpha=0.3, prec=prec, refine_iters=4,
                        refine_tol=1e-13, phase=ph)
    assert np.max(np.abs(U.cpu().numpy() - U1)) < 1e-10
    assert np.max(np.abs(D.cpu().numpy() - D1)) < 1e-10
    assert abs(dn - np.max(np.abs(n1))) < 1e-10
    assert np.max(np.abs(n_prev.cpu().numpy() - n1)) < 1e-10
