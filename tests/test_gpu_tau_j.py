"""Parity of bdg_kinetic_current_densities (tau and j of the densities equation) with the FP64
oracle.  Both sides take the oracle's eigenpairs, so the comparison isolates the densities:
vortex states, finite temperature, a grid dimension of one point, and a real state without
current."""
import numpy as np
import pytest

import oracle
import workloads as wk
from tests.gpu_common import ctx, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,nv,T", [((6, 4, 4), 1, 0.0), ((4, 4, 6), 2, 0.1), ((6, 4, 1), 1, 0.0),
                                        ((4, 6, 2), 0, 0.05)])
def test_tau_and_current_match_oracle(shape, nv, T):
    import paper_2310_03341_b300 as bdg
    w = wk.random_small(*shape, seed=5, n_vortices=nv)
    ew, Zo = oracle.heev(oracle.build(w))
    tau_o, j_o = oracle.kinetic_current_densities(ew, Zo, shape, T=T)
    evt = torch.tensor(ew, device="cuda")
    Zt = bdg.colmajor(torch.tensor(Zo, device="cuda"))
    tau, j = ctx().kinetic_current_densities(shape, evt, Zt, T=T)
    tau, j = tau.cpu().numpy(), j.cpu().numpy()
    scale = np.max(np.abs(tau_o))
    assert np.max(np.abs(tau - tau_o)) <= 1e-12 * scale
    assert np.max(np.abs(j - j_o)) <= 1e-12 * scale
    if nv == 0:
        assert np.max(np.abs(j)) <= 1e-14 * scale
