"""bdg_densities_noalloc against bdg_densities.

Some callers cannot allocate device memory inside their self-consistent loop:
a host application whose own allocator already holds the device memory it may
use, or a loop that must not take the device-wide synchronisation that
cudaFree implies.  bdg_densities_noalloc serves them: it keeps its scratch in
a fixed device array of the library instead of a context workspace.

These tests call it through the C ABI (the binding only marshals arguments)
two times in a row on different grids and temperatures, compare each result
with bdg_densities on the same eigenpairs, check that the device's free memory
does not move across calls once the first call has set up the scratch address,
and check that a grid beyond the scratch limit is refused before any launch.
Two grids are large enough that the scratch size, not the device's SM count,
caps the number of column chunks: V = 3840 (45 chunks) and V = 172800, next to
the largest accepted grid (one chunk, 4.15 of the 4.19 MB scratch in use).
The file is named to be collected last, so it also runs after every other GPU
test in the same process.
"""
import numpy as np
import pytest

import workloads as wk
from tests.gpu_common import ctx, dev_fields, torch

pytestmark = pytest.mark.gpu


def _eigpairs(w):
    U, D = dev_fields(w)
    c = ctx()
    H = c.build((w.nx, w.ny, w.nz), w.mu, U, D)
    ev, Z = c.heev(H, "fp64", overwrite=True)
    return ev, Z


def _random_pairs(V, ncols, window, seed):
    """Seeded sorted eigenvalues with `window` of them in (0, Ec) at the front and the
    rest above Ec, and a column-major Z (2V rows) holding `ncols` random columns.  The
    densities read only the window's columns, so Z needs no more than those."""
    import math
    rng = np.random.default_rng(seed)
    Ec = math.pi ** 2 / 2
    n = 2 * V
    w = np.sort(np.concatenate([rng.uniform(0.05, Ec - 0.05, window), rng.uniform(Ec + 0.1, Ec + 5, n - window)]))
    Zb = torch.empty(ncols, n, dtype=torch.complex128, device="cuda")
    g = torch.Generator(device="cuda").manual_seed(seed)
    Zb.real.normal_(generator=g)
    Zb.imag.normal_(generator=g)
    Zb /= np.sqrt(n)
    return torch.tensor(w, dtype=torch.float64, device="cuda"), Zb.mT


def _compare(nd, nu, nd_ref, nu_ref, rel):
    assert torch.isfinite(nd).all() and torch.isfinite(torch.view_as_real(nu)).all()
    sn = max(torch.max(torch.abs(nd_ref)).item(), 1e-300)
    snu = max(torch.max(torch.abs(nu_ref)).item(), 1e-300)
    assert torch.max(torch.abs(nd - nd_ref)).item() <= rel * sn
    assert torch.max(torch.abs(nu - nu_ref)).item() <= rel * snu


def test_noalloc_matches_bdg_densities_on_two_calls_in_a_row():
    import paper_2310_03341_b300 as bdg
    cases = [(wk.random_small(4, 4, 6, seed=11, n_vortices=1), 0.0),
             (wk.random_small(6, 6, 8, seed=12, n_vortices=2), 0.05)]
    pairs = [_eigpairs(w) for w, _ in cases]
    refs = [ctx().densities((w.nx, w.ny, w.nz), ev, Z, T=T) for (w, T), (ev, Z) in zip(cases, pairs)]
    outs = [(torch.empty(w.V, dtype=torch.float64, device="cuda"),
             torch.empty(w.V, dtype=torch.complex128, device="cuda")) for w, _ in cases]
    torch.cuda.synchronize()

    def run():
        for (w, T), (ev, Z), (nd, nu) in zip(cases, pairs, outs):
            nd.fill_(np.nan)
            nu.fill_(np.nan)
            bdg.densities_noalloc((w.nx, w.ny, w.nz), ev, Z, nd, nu, T=T)
        torch.cuda.synchronize()

    run()      # the first call on this device sets up the scratch address
    free0 = torch.cuda.mem_get_info()[0]
    run()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0
    for (nd_ref, nu_ref), (nd, nu) in zip(refs, outs):
        assert torch.isfinite(nd).all() and torch.isfinite(torch.view_as_real(nu)).all()
        assert torch.max(torch.abs(nd - nd_ref)).item() <= 1e-14
        assert torch.max(torch.abs(nu - nu_ref)).item() <= 1e-14


@pytest.mark.parametrize("grid,ncols,window,T", [((12, 16, 20), None, 900, 0.0),
                                                 ((40, 40, 108), 16, 16, 0.02)])
def test_noalloc_where_the_scratch_caps_the_chunks(grid, ncols, window, T):
    """V = 3840: 45 chunks fit the scratch (the SM count alone would give 64);
    V = 172800: one chunk, close to the largest accepted grid.  Two calls in a row."""
    import paper_2310_03341_b300 as bdg
    V = grid[0] * grid[1] * grid[2]
    n = 2 * V
    ev, Z = _random_pairs(V, n if ncols is None else ncols, window, seed=V)
    nd_ref, nu_ref = ctx().densities(grid, ev, Z, T=T)
    for _ in range(2):
        nd = torch.full((V,), np.nan, dtype=torch.float64, device="cuda")
        nu = torch.full((V,), np.nan, dtype=torch.complex128, device="cuda")
        bdg.densities_noalloc(grid, ev, Z, nd, nu, T=T)
        torch.cuda.synchronize()
        _compare(nd, nu, nd_ref, nu_ref, 1e-13)


def test_noalloc_refuses_grids_beyond_the_scratch_limit():
    import paper_2310_03341_b300 as bdg
    grid = (56, 56, 56)                      # V = 175616 > 174720
    V = 56 ** 3
    w = torch.zeros(2 * V, dtype=torch.float64, device="cuda")
    Z = torch.zeros(1, 2 * V, dtype=torch.complex128, device="cuda").mT
    nd = torch.zeros(V, dtype=torch.float64, device="cuda")
    nu = torch.zeros(V, dtype=torch.complex128, device="cuda")
    with pytest.raises(bdg.BdgError) as e:
        bdg.densities_noalloc(grid, w, Z, nd, nu)
    assert e.value.code == -6
    assert "scratch limit" in str(e.value)


def test_noalloc_refuses_an_odd_grid_like_bdg_densities():
    import paper_2310_03341_b300 as bdg
    grid = (4, 3, 4)
    V = 48
    w = torch.zeros(2 * V, dtype=torch.float64, device="cuda")
    Z = torch.zeros(2 * V, 2 * V, dtype=torch.complex128, device="cuda").mT
    nd = torch.zeros(V, dtype=torch.float64, device="cuda")
    nu = torch.zeros(V, dtype=torch.complex128, device="cuda")
    with pytest.raises(bdg.BdgError) as e:
        bdg.densities_noalloc(grid, w, Z, nd, nu)
    assert e.value.code == -1
    with pytest.raises(bdg.BdgError) as e2:
        ctx().densities(grid, w, Z)
    assert e2.value.code == -1
