"""Host-side set-up of the learned SCF guess against the oracle (no GPU)."""
import numpy as np

import oracle
from paper_2310_03341_b300 import fno


def test_coupling_for_gap_matches_the_oracle():
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
