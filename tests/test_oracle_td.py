"""Pins of the time-evolution oracle (oracle/tdslda.py): the quasiparticle wavefunctions
of Eq. (TDSLDA) stepped with the fifth-order Adams-Bashforth-Moulton predictor-corrector.

* Linear case (g = 0): H does not depend on time and the exact propagator is
  Z exp(-i Lambda t) Z^H with numpy's dense eigendecomposition; the error falls as dt^5.
* A self-consistent stationary state (the uniform gap-equation state, complex gap) only
  turns its phases: phi_n(t) = phi_n(0) exp(-i E_n t), the densities stay put.
* Any state stays orthonormal (the evolution is unitary), and a state that is not
  self-consistent does move (the density-dependent H is live).
Planted mistakes (a wrong predictor weight, a conjugated nu, a flipped Hartree sign, a
dropped -i) make one of these fail."""
import numpy as np
import pytest

import oracle
import oracle.tdslda as td
import workloads as wk


def _window(w):
    ev, Z = np.linalg.eigh(oracle.build(w))
    sel = np.nonzero((ev > 0) & (ev < np.pi ** 2 / 2))[0]
    return ev[sel], Z[:, sel]


def _linear_case():
    w = wk.random_small(4, 4, 2, seed=3, n_vortices=1)
    rng = np.random.default_rng(5)
    X = rng.standard_normal((w.N, 6)) + 1j * rng.standard_normal((w.N, 6))
    Psi0, _ = np.linalg.qr(X)
    return w, Psi0


def _exact_linear(w, Psi0, t):
    # g = 0: U = U_ext, Delta = 0 -> H(U_ext, 0); exact propagator from numpy's eigh
    wl = wk.Workload("lin", w.nx, w.ny, w.nz, w.mu, w.U, np.zeros(w.V, complex), {})
    lam, Zh = np.linalg.eigh(oracle.build(wl))
    return Zh @ (np.exp(-1j * lam * t)[:, None] * (Zh.conj().T @ Psi0))


def test_linear_case_matches_the_exact_propagator_at_fifth_order():
    w, Psi0 = _linear_case()
    E0 = np.full(Psi0.shape[1], 1.0)
    ref = _exact_linear(w, Psi0, 1.0)
    errs = []
    for dt in (0.01, 0.005):
        Psi, _, _ = td.evolve((w.nx, w.ny, w.nz), w.mu, 0.0, Psi0, E0, dt, int(round(1.0 / dt)), U_ext=w.U)
        errs.append(np.max(np.abs(Psi - ref)))
    assert errs[0] < 1e-5
    assert 24.0 < errs[0] / errs[1] < 42.0           # 2^5 = 32 (measured 34.6)


def _stationary_case():
    nx, ny, nz, mu = 4, 4, 4, 0.5
    d0 = 0.3 * np.exp(0.7j)
    g, U0 = oracle.gap_coupling(nx, ny, nz, mu, abs(d0))
    w = wk.uniform(nx, ny, nz, mu, U0, 0.0)
    w.Delta = np.full(w.V, d0, dtype=np.complex128)
    E0, Psi0 = _window(w)
    return w, g, E0, Psi0


def test_self_consistent_state_only_turns_its_phases():
    w, g, E0, Psi0 = _stationary_case()
    t, dt = 1.0, 0.02
    Psi, n, nu = td.evolve((w.nx, w.ny, w.nz), w.mu, g, Psi0, E0, dt, int(round(t / dt)))
    assert np.max(np.abs(Psi - Psi0 * np.exp(-1j * E0 * t)[None, :])) < 1e-6
    n0, nu0 = td.densities(Psi0, w.V, *td.weights(E0, 0.0))
    assert np.max(np.abs(n - n0)) < 1e-8 and np.max(np.abs(nu - nu0)) < 1e-8
    assert np.max(np.abs(g * nu0 - w.Delta)) < 1e-12    # the state really is self-consistent


def _moving_case():
    w = wk.random_small(4, 4, 4, seed=2, n_vortices=1)
    g, _ = oracle.gap_coupling(w.nx, w.ny, w.nz, w.mu, 0.3)
    E0, Psi0 = _window(w)
    return w, g, E0, Psi0


def test_evolution_is_unitary_and_the_density_dependent_hamiltonian_acts():
    w, g, E0, Psi0 = _moving_case()
    Psi, n, nu = td.evolve((w.nx, w.ny, w.nz), w.mu, g, Psi0, E0, 0.02, 25, U_ext=w.U)
    G = Psi.conj().T @ Psi
    assert np.max(np.abs(G - np.eye(G.shape[0]))) < 1e-6     # integration error (measured 1.8e-7)
    n0, nu0 = td.densities(Psi0, w.V, *td.weights(E0, 0.0))
    assert np.max(np.abs(n - n0)) > 1e-3              # not a stationary state of the live H


# ---- planted mistakes -------------------------------------------------------------------
def test_a_wrong_predictor_weight_breaks_the_order(monkeypatch):
    monkeypatch.setattr(td, "AB5", td.AB5 * np.array([1.0, 1.0, 1.0, 1.0, 0.5]))
    w, Psi0 = _linear_case()
    E0 = np.full(Psi0.shape[1], 1.0)
    ref = _exact_linear(w, Psi0, 1.0)
    errs = [np.max(np.abs(td.evolve((w.nx, w.ny, w.nz), w.mu, 0.0, Psi0, E0, dt, int(round(1.0 / dt)),
                                    U_ext=w.U)[0] - ref)) for dt in (0.01, 0.005)]
    assert not (errs[0] < 1e-5 and 24.0 < errs[0] / errs[1] < 42.0)


def test_a_dropped_minus_i_breaks_the_linear_case(monkeypatch):
    orig = td.rhs
    monkeypatch.setattr(td, "rhs", lambda *a, **k: 1j * orig(*a, **k))   # +i instead of -i: time reversed
    w, Psi0 = _linear_case()
    E0 = np.full(Psi0.shape[1], 1.0)
    Psi, _, _ = td.evolve((w.nx, w.ny, w.nz), w.mu, 0.0, Psi0, E0, 0.02, 50, U_ext=w.U)
    assert np.max(np.abs(Psi - _exact_linear(w, Psi0, 1.0))) > 1e-2


@pytest.mark.parametrize("mistake", ["conj_nu", "hartree_sign"])
def test_functional_mistakes_break_the_stationary_state(monkeypatch, mistake):
    if mistake == "conj_nu":
        orig = td.densities
        monkeypatch.setattr(td, "densities", lambda *a: (orig(*a)[0], np.conj(orig(*a)[1])))
    else:
        monkeypatch.setattr(td, "fields", lambda n, nu, g, U_ext: (0.5 * g * n, g * nu))
    w, g, E0, Psi0 = _stationary_case()
    Psi, _, _ = td.evolve((w.nx, w.ny, w.nz), w.mu, g, Psi0, E0, 0.02, 50)
    assert np.max(np.abs(Psi - Psi0 * np.exp(-1j * E0 * 1.0)[None, :])) > 1e-3
