"""Plausible mistakes planted in a copy of the FNO reference must fail its pins."""
import numpy as np
import pytest

from oracle import fno
from tests import test_oracle_fno as pins


def test_flipped_transform_sign_is_caught(monkeypatch):
    monkeypatch.setattr(fno.np.fft, "fftn", np.fft.ifftn)
    monkeypatch.setattr(fno.np.fft, "ifftn", np.fft.fftn)
    with pytest.raises(AssertionError):
        pins.test_plane_wave_through_one_complex_mode_fixes_the_transform_convention()


def test_mode_order_reversal_is_caught(monkeypatch):
    real = fno.mode_indices
    monkeypatch.setattr(fno, "mode_indices", lambda g, m: tuple(a[::-1] for a in real(g, m)))
    with pytest.raises(AssertionError):
        pins.test_plane_wave_through_one_complex_mode_fixes_the_transform_convention()


def test_dropped_low_pass_mask_is_caught(monkeypatch):
    """Keeping every mode (no truncation) must fail the low-pass pin."""
    monkeypatch.setattr(fno, "mode_indices", lambda g, m: tuple(
        a.ravel() for a in np.meshgrid(np.arange(g), np.arange(g), np.arange(g), indexing="ij")))
    with pytest.raises(Exception):
        pins.test_spectral_layer_with_identity_modes_is_a_low_pass_filter()


def test_missing_gelu_is_caught(monkeypatch):
    monkeypatch.setattr(fno, "gelu", lambda x: x)
    with pytest.raises(AssertionError):
        pins.test_zero_spectral_weights_reduce_to_a_pointwise_mlp()
