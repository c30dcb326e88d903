"""Batched kz-block solver (bdg_heev_batched) against the FP64 oracle.

A z-invariant system splits exactly into kz blocks H_kz = H_perp + (kz^2/2)
tau_z; the union of the block spectra is the spectrum of the full 3-D
matrix.  Blocks of uneven sizes are solved concurrently by the worker pool,
including size classes large enough to trigger the band-width autotuner."""
import numpy as np
import pytest

import oracle
import workloads as wk
from tests import pins
from tests.gpu_common import ctx, torch

pytestmark = pytest.mark.gpu


def _z_invariant(nx, ny, nz, seed):
    """2-D fields (vortex + smooth U) replicated along z."""
    D2 = wk.vortex_pairing(nx, ny, 1, 0.3, [(0.3, -0.2)], [1])
    U2 = -0.4 + wk.smooth_field((nx, ny), 2.0, seed, 0.05)
    U3 = np.repeat(U2.reshape(nx * ny), nz)        # site (ix, iy, iz): z fastest
    D3 = np.repeat(D2.reshape(nx * ny), nz)
    return U2, D2, wk.Workload(f"zinv_{nx}x{ny}x{nz}", nx, ny, nz, 0.5, U3, D3, {})


def _kz(nz):
    return [2 * np.pi * m / nz for m in range(-nz // 2, nz // 2)]


@pytest.mark.parametrize("prec", ["fp64", "bf16x9"])
def test_union_of_kz_block_spectra_is_the_3d_spectrum(prec):
    nx, ny, nz = 6, 6, 8
    U2, D2, w3 = _z_invariant(nx, ny, nz, seed=7)
    ew = oracle.heev(oracle.build(w3), vectors=False)
    c = ctx()
    blocks = c.build_kz_blocks((nx, ny), w3.mu, torch.tensor(U2.reshape(-1), device="cuda"),
                               torch.tensor(D2.reshape(-1), device="cuda"), _kz(nz))
    res = c.heev_batched(blocks, prec, ph=True)
    union = np.sort(np.concatenate([r[0].cpu().numpy() for r in res]))
    rho = np.max(np.abs(ew))
    assert np.max(np.abs(union - ew)) / rho <= (1e-12 if prec == "fp64" else 1e-5)


def test_plus_and_minus_kz_blocks_have_equal_spectra():
    nx, ny, nz = 6, 4, 8
    U2, D2, w3 = _z_invariant(nx, ny, nz, seed=8)
    kz = _kz(nz)
    c = ctx()
    blocks = c.build_kz_blocks((nx, ny), w3.mu, torch.tensor(U2.reshape(-1), device="cuda"),
                               torch.tensor(D2.reshape(-1), device="cuda"), kz)
    res = c.heev_batched(blocks, "fp64")
    ev = {round(k, 12): r[0].cpu().numpy() for k, r in zip(kz, res)}
    rho = max(np.max(np.abs(v)) for v in ev.values())
    for k in kz:
        if k > 0:
            assert np.max(np.abs(ev[round(k, 12)] - ev[round(-k, 12)])) / rho <= 1e-13


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x9"])
def test_uneven_blocks_match_oracle(prec):
    """Sizes 32 .. 200 with a class of 6 blocks (autotuned band) and singletons."""
    shapes = [(4, 4), (6, 6), (10, 10), (8, 6)] + [(8, 8)] * 6
    c = ctx()
    blocks, mats, ws = [], [], []
    for i, (nx, ny) in enumerate(shapes):
        w = wk.random_small(nx, ny, 1, seed=20 + i, n_vortices=1)
        U = torch.tensor(w.U, device="cuda")
        D = torch.tensor(w.Delta, device="cuda")
        blocks.append(c.build((nx, ny, 1), w.mu, U, D))
        mats.append(oracle.build(w))
        ws.append(w)
    res = c.heev_batched(blocks, prec)
    tol_e, tol_r = (1e-12, 1e-12) if prec == "fp64" else (1e-5, 1e-4)
    for H, w, (ev, Z) in zip(mats, ws, res):
        ev, Z = ev.cpu().numpy(), Z.cpu().numpy()
        ew = oracle.heev(H, vectors=False)
        rho = np.max(np.abs(ew))
        assert np.max(np.abs(ev - ew)) / rho <= tol_e
        assert np.max(np.linalg.norm(H @ Z - Z * ev, axis=0)) / rho <= tol_r
        assert oracle.orthogonality(Z) <= (1e-10 if prec == "fp64" else 1e-4)


def test_uniform_tube_closed_form():
    """Uniform U = 0, Delta0 on an 8 x 8 cross-section: E = +-sqrt((k_perp^2/2 + kz^2/2 - mu)^2 + Delta0^2)."""
    nx, ny, nz, mu, D0 = 8, 8, 8, 0.5, 0.2
    kz = _kz(nz)
    c = ctx()
    U = torch.zeros(nx * ny, dtype=torch.float64, device="cuda")
    D = torch.full((nx * ny,), D0, dtype=torch.complex128, device="cuda")
    res = c.heev_batched(c.build_kz_blocks((nx, ny), mu, U, D, kz), "fp64", ph=True)
    for k, (ev, _) in zip(kz, res):
        ref = pins.uniform_spectrum(nx, ny, 1, mu - 0.5 * k * k, 0.0, D0)
        assert np.max(np.abs(ev.cpu().numpy() - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_build_with_a_size_one_dimension_matches_oracle():
    w = wk.random_small(6, 4, 1, seed=31, n_vortices=1)
    H = ctx().build((w.nx, w.ny, w.nz), w.mu, torch.tensor(w.U, device="cuda"),
                    torch.tensor(w.Delta, device="cuda")).cpu().numpy()
    Ho = oracle.build(w)
    assert np.max(np.abs(H - Ho)) < 1e-14 * max(1.0, np.max(np.abs(Ho)))
