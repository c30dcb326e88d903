"""bdg_densities_noalloc against bdg_densities.

The allocation-free entry point keeps its scratch in a fixed device array of
the library instead of a context workspace.  These tests run two calls in a
row on different grids and temperatures, compare each with bdg_densities on
the same eigenpairs, check that the device's free memory does not move across
calls once the first call has set up the scratch address, and check that a
grid beyond the scratch limit is refused before any launch.  The file is
named to be collected last, so it also runs after every other GPU test in
the same process.
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


def test_noalloc_refuses_grids_beyond_the_scratch_limit():
    import paper_2310_03341_b300 as bdg
    w = torch.zeros(4, dtype=torch.float64, device="cuda")
    Z = torch.zeros(4, 4, dtype=torch.complex128, device="cuda").mT
    nd = torch.zeros(2, dtype=torch.float64, device="cuda")
    nu = torch.zeros(2, dtype=torch.complex128, device="cuda")
    with pytest.raises(bdg.BdgError) as e:
        bdg.densities_noalloc((56, 56, 56), w, Z, nd, nu)   # V = 175616 > 174720
    assert e.value.code == -6
    assert "scratch limit" in str(e.value)
