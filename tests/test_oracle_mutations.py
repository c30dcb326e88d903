"""Planted mistakes: each variant of the oracle (built here, on the CPU) has a
plausible error, and at least one pin must reject it.  This shows the pins
have the power to catch a dropped term, a wrong sign, a transposed block, a
broken reduction step, swapped or conjugated density terms, a broken Fermi
weight or a wrong sign in the self-consistent update."""
import numpy as np
import pytest

import workloads as wk
from tests import pins


def _mut_build(orc, kind):
    def build(w):
        H = orc.build(w)
        V = w.V
        if kind == "no_mu":
            H[np.arange(V), np.arange(V)] += w.mu
            H[V + np.arange(V), V + np.arange(V)] -= w.mu
        elif kind == "lower_block_sign":
            H[V:, V:] = H[:V, :V]
        elif kind == "delta_blocks_swapped":
            H[np.arange(V), V + np.arange(V)] = np.conj(w.Delta)
            H[V + np.arange(V), np.arange(V)] = w.Delta
        elif kind == "kinetic_factor":
            h = H[:V, :V].copy()
            diag = np.diag(np.diag(h))
            H[:V, :V] = 2 * (h - diag) + diag
            H[V:, V:] = -H[:V, :V].conj()
        elif kind == "nyquist_dropped":
            H = H.copy()
            # remove the m = -n/2 term of every 1-D kinetic matrix
            ix, iy, iz = np.meshgrid(np.arange(w.nx), np.arange(w.ny), np.arange(w.nz), indexing="ij")
            ix, iy, iz = ix.ravel(), iy.ravel(), iz.ravel()
            for a, n in ((ix, w.nx), (iy, w.ny), (iz, w.nz)):
                others = [b for b in (ix, iy, iz) if b is not a]
                same = (others[0][:, None] == others[0][None, :]) & (others[1][:, None] == others[1][None, :])
                corr = (np.pi ** 2 / 2) * (-1.0) ** (a[:, None] - a[None, :]) / n
                H[:V, :V] -= same * corr
                H[V:, V:] += same * corr
        return H
    return build


def _mut_heev(orc, kind):
    def heev(H, vectors=False):
        d, e, tau, _ = orc.tridiag(H)
        if kind == "phase_real_part":
            er = np.real(e)
        elif kind == "offdiag_scaled":
            er = np.abs(e) * (1 - 1e-6)
        elif kind == "last_offdiag_dropped":
            er = np.abs(e)
            er[-1] = 0.0
        return orc.tqr(d, er)
    return heev


@pytest.mark.parametrize("kind", ["no_mu", "lower_block_sign", "kinetic_factor", "nyquist_dropped"])
def test_uniform_pin_rejects_broken_build(orc, kind):
    with pytest.raises(AssertionError):
        pins.check_uniform(_mut_build(orc, kind), orc.heev, 4, 4, 4)


def test_phase_pin_rejects_swapped_pairing_blocks(orc):
    w = wk.random_small(6, 6, 4, seed=9, n_vortices=1, amplitude=0.4)
    pins.check_pairing_phase(orc.build, orc.heev, orc.densities, w)
    with pytest.raises(AssertionError):
        pins.check_pairing_phase(_mut_build(orc, "delta_blocks_swapped"), orc.heev, orc.densities, w)


@pytest.mark.parametrize("kind", ["phase_real_part", "offdiag_scaled", "last_offdiag_dropped"])
def test_lapack_pin_rejects_broken_reduction(orc, kind):
    w = wk.random_small(4, 4, 6, seed=1, n_vortices=2)
    pins.check_vs_lapack(orc.build, lambda H, vectors=False: orc.heev(H, vectors=False), w)
    with pytest.raises(AssertionError):
        pins.check_vs_lapack(orc.build, _mut_heev(orc, kind), w)


def test_frobenius_pin_rejects_broken_build(orc):
    w = wk.random_small(4, 4, 4, seed=2)
    with pytest.raises(AssertionError):
        pins.check_frobenius_and_trace(_mut_build(orc, "kinetic_factor"), w)
    with pytest.raises(AssertionError):
        pins.check_frobenius_and_trace(_mut_build(orc, "no_mu"), w)


def _mut_densities(orc, kind):
    def densities(ev, Z, V, T=0.0):
        if kind == "u_v_swapped":
            return orc.densities(ev, np.concatenate([Z[V:], Z[:V]]), V, T=T)
        n, nu = orc.densities(ev, Z, V, T=T)
        if kind == "spin_factor_dropped":
            return n / 2, nu
        if kind == "nu_conjugated":
            return n, np.conj(nu)
        return n, nu
    return densities


@pytest.mark.parametrize("kind", ["u_v_swapped", "spin_factor_dropped"])
def test_density_pin_rejects_broken_sums(orc, kind):
    with pytest.raises(AssertionError):
        pins.check_uniform_densities(orc.build, orc.heev, _mut_densities(orc, kind), 4, 4, 6)


def test_phase_pin_rejects_conjugated_nu(orc):
    w = wk.random_small(6, 6, 4, seed=9, n_vortices=1, amplitude=0.4)
    with pytest.raises(AssertionError):
        pins.check_pairing_phase(orc.build, orc.heev, _mut_densities(orc, "nu_conjugated"), w)


@pytest.mark.parametrize("kind", ["sign", "temperature_scale"])
def test_finite_temperature_pin_rejects_broken_fermi(orc, monkeypatch, kind):
    """The mistake is planted in the oracle's own Fermi function, which its densities call."""
    good = orc.fermi
    bad = {"sign": lambda E, T: good(-np.asarray(E), T),
           "temperature_scale": lambda E, T: good(E, 0.5 * T)}[kind]
    monkeypatch.setattr(orc, "fermi", bad)
    with pytest.raises(AssertionError):
        pins.check_uniform_densities(orc.build, orc.heev, orc.densities, 4, 4, 6, T=0.05)


def _mut_scf(orc, kind):
    def scf_step(w, g, alpha=0.3):
        U1, D1, n, nu = orc.scf_step(w, g, alpha=alpha)
        if kind == "hartree_sign":
            U1 = (1 - alpha) * w.U + alpha * (g * n / 2.0)
        elif kind == "delta_conjugated":
            D1 = (1 - alpha) * w.Delta + alpha * g * np.conj(nu)
        return U1, D1, n, nu
    return scf_step


def test_fixed_point_pin_rejects_hartree_sign(orc):
    with pytest.raises(AssertionError):
        pins.check_scf_fixed_point(_mut_scf(orc, "hartree_sign"), orc.gap_coupling, 4, 4, 4)


def test_scf_phase_pin_rejects_conjugated_update(orc):
    w = wk.random_small(6, 6, 4, seed=9, n_vortices=1, amplitude=0.4)
    g, _ = orc.gap_coupling(6, 6, 4, w.mu, 0.4)
    with pytest.raises(AssertionError):
        pins.check_scf_phase(_mut_scf(orc, "delta_conjugated"), w, g)


def _mut_kcd(orc, kind):
    def kcd(ev, Z, shape, T=0.0):
        if kind == "tau_weights_swapped":      # |grad v|^2 weighted by f(E), |grad u|^2 by f(-E)
            V = int(np.prod(shape))
            tau, j = orc.kinetic_current_densities(ev, np.concatenate([Z[V:], Z[:V]]), shape, T=T)
            return tau, j
        tau, j = orc.kinetic_current_densities(ev, Z, shape, T=T)
        if kind == "tau_factor_dropped":
            return tau / 2, j
        if kind == "current_sign":
            return tau, -j
        return tau, j
    return kcd


@pytest.mark.parametrize("kind", ["tau_weights_swapped", "tau_factor_dropped"])
def test_tau_pin_rejects_broken_kinetic_density(orc, kind):
    with pytest.raises(AssertionError):
        pins.check_uniform_tau(orc.build, orc.heev, _mut_kcd(orc, kind), 4, 4, 6)


def test_boost_and_vortex_pins_reject_a_flipped_current(orc):
    with pytest.raises(AssertionError):
        pins.check_boost_current(orc.build, orc.heev, orc.densities, _mut_kcd(orc, "current_sign"))
    with pytest.raises(AssertionError):
        pins.check_vortex_circulation(orc.build, orc.heev, _mut_kcd(orc, "current_sign"), 1)


def test_uniform_pin_rejects_a_current_gradient_with_the_nyquist_mode(orc, monkeypatch):
    """Keeping k = -pi in the current's gradient makes the real plane wave (-1)^x carry a
    spurious current; the mistake is planted in the oracle's own gradient."""
    good = orc.spectral_gradient
    monkeypatch.setattr(orc, "spectral_gradient", lambda F, shape, keep_nyquist: good(F, shape, True))
    with pytest.raises(AssertionError):
        pins.check_uniform_tau(orc.build, orc.heev, orc.kinetic_current_densities, 4, 4, 6)
