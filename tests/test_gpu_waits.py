"""Bounded device waits, made to run out on purpose.

Every device-side wait of the library has a cap (bdg_set_wait_limit): the
tensor-core pipeline barriers and the stage-2 wait of a sweep on its
predecessor.  With a cap of a few clock cycles a wait gives up; the kernel
sets the context's error word, drains what it has in flight and returns, and
the call reports BDG_ETIMEOUT.  Nothing faults or hangs: the failure is a
status the host reads.  The next call on the same context, with the default
cap restored, must again match the oracle."""
import numpy as np
import pytest

import oracle
import workloads as wk
from tests.gpu_common import dev_fields, torch

pytestmark = pytest.mark.gpu


def _solve(c, w, prec):
    U, D = dev_fields(w)
    grid = (w.nx, w.ny, w.nz)
    H = c.build(grid, w.mu, U, D)
    ev, Z = c.heev(H, prec, overwrite=True, ph=True)
    return U, D, ev, Z


@pytest.mark.parametrize("prec", ["bf16x9", "fp64"])
def test_capped_waits_time_out_and_the_context_recovers(prec):
    import paper_2310_03341_b300 as bdg
    w = wk.random_small(4, 6, 10, seed=1, n_vortices=2)     # N = 480: several panels and sweeps
    c = bdg.Context(0)
    try:
        c.set_wait_limit(8)
        with pytest.raises(bdg.BdgError) as e:
            _solve(c, w, prec)
        assert e.value.code == bdg.ERRORS_BY_NAME["ETIMEOUT"]
        torch.cuda.synchronize()
        c.set_wait_limit(0)
        U, D, ev, Z = _solve(c, w, prec)
        if prec != "fp64":
            _, _, _, ok = c.refine((w.nx, w.ny, w.nz), w.mu, U, D, ev, Z, 6, 1e-12)
            assert ok
        torch.cuda.synchronize()
        ew, _ = oracle.heev(oracle.build(w))
        rho = float(np.max(np.abs(ew)))
        evh, Zh = ev.cpu().numpy(), Z.cpu().numpy()
        assert np.max(np.abs(evh - ew)) / rho <= 1e-12
        assert np.max(oracle.residuals(w, evh, Zh)) / rho <= 1e-11
    finally:
        c.close()


def test_wait_limit_rejects_negative_caps():
    import paper_2310_03341_b300 as bdg
    c = bdg.Context(0)
    try:
        with pytest.raises(bdg.BdgError):
            c.set_wait_limit(-1)
    finally:
        c.close()
