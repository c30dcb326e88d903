"""Host-side set-up of the learned SCF guess against the oracle (no GPU)."""
import numpy as np

import oracle
from paper_2310_03341_b300 import fno


def test_coupling_for_gap_matches_the_oracle():
    """bdg_gap_coupling (host arithmetic inside the library) against the oracle's gap equation on
    8^3 grids and on scaled coarse levels (dx = 1.5 and 2: mu and Delta0 times s = dx^2); a gap
    above the cutoff leaves no state in the window and is refused."""
    import pytest
    import paper_2310_03341_b300 as bdg
    for s in (2.25, 4.0):
        g1, U1 = bdg.gap_coupling((4, 4, 2), s * 0.5, s * 0.45)
        g2, U2 = oracle.gap_coupling(4, 4, 2, s * 0.5, s * 0.45)
        assert abs(g1 - g2) <= 1e-10 * g2 and abs(U1 - U2) <= 1e-10 * abs(U2)
    with pytest.raises(bdg.BdgError):
        bdg.gap_coupling((4, 4, 2), 16 * 0.5, 16 * 0.45)
    for seed in range(6):
        w = fno.sample(seed, 8)
        g1, U1 = fno.coupling_for_gap(8, 8, 8, w.mu, w.meta["Delta0"])
        g2, U2 = oracle.gap_coupling(8, 8, 8, w.mu, w.meta["Delta0"])
        assert abs(g1 - g2) <= 1e-10 * g2 and abs(U1 - U2) <= 1e-10


def test_features_describe_the_ansatz():
    w = fno.sample(3, 8)
    f = fno.features(w)
    assert f.shape == (w.V, 5)
    d = f[:, 2] * (f[:, 3] + 1j * f[:, 4]) * w.meta["Delta0"]
    assert np.max(np.abs(d - w.Delta)) < 1e-6
