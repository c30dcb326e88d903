"""Pins of the FP64 CPU oracle (no GPU): closed forms, invariants, LAPACK."""
import numpy as np
import pytest
import scipy.linalg

import workloads as wk
from tests import pins


@pytest.mark.parametrize("n", [2, 4, 6, 8, 16, 24, 32])
def test_kinetic_matrix_definition(orc, n):
    """The DFT-sum kinetic matrix equals the closed-form circulant, has spectrum
    {k^2/2}, and acts like F^-1 (k^2/2) F (numpy FFT)."""
    T, im = orc.kinetic_1d(n)
    assert im < 1e-12
    assert np.max(np.abs(T - T.T)) < 1e-13
    col = pins.closed_form_kinetic_column(n)
    for b in range(n):
        idx = (np.arange(n) - b) % n
        assert np.max(np.abs(T[:, b] - col[idx])) < 1e-12 * np.pi ** 2
    k = 2 * np.pi * np.arange(-n // 2, n // 2) / n
    assert np.max(np.abs(np.linalg.eigvalsh(T) - np.sort(k * k / 2))) < 1e-12
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    kf = 2 * np.pi * np.fft.fftfreq(n)
    kf[np.isclose(kf, np.pi)] = -np.pi          # Nyquist mode is -pi (n = -N/2)
    y = np.fft.ifft(0.5 * kf ** 2 * np.fft.fft(x))
    assert np.max(np.abs(T @ x - y)) < 1e-12


def test_build_structure(orc):
    w = wk.random_small(4, 4, 6, seed=3)
    H = orc.build(w)
    V = w.V
    assert np.max(np.abs(H - H.conj().T)) == 0.0
    assert np.max(np.abs(H[V:, V:] + H[:V, :V].conj())) == 0.0
    assert np.max(np.abs(H[:V, V:] - np.diag(w.Delta))) == 0.0
    assert np.max(np.abs(H[V:, :V] - np.diag(w.Delta.conj()))) == 0.0
    pins.check_frobenius_and_trace(orc.build, w)


@pytest.mark.parametrize("shape", [(4, 4, 4), (4, 6, 8), (2, 4, 6)])
def test_uniform_closed_form(orc, shape):
    pins.check_uniform(orc.build, orc.heev, *shape)


def test_uniform_c1_closed_form_and_vectors(orc):
    """Config C1 (uniform 8^3, N=1024): all eigenpairs against the closed form."""
    w = wk.c1_uniform()
    H = orc.build(w)
    ev, Z = orc.heev(H)
    ref = pins.uniform_spectrum(8, 8, 8, 0.5, 0.0, 0.2)
    rho = np.max(np.abs(ref))
    assert np.max(np.abs(ev - ref)) / rho < 1e-13
    res = orc.residuals(w, ev, Z)
    assert np.max(res) / rho < 1e-13
    assert orc.orthogonality(Z) < 1e-12


@pytest.mark.parametrize("shape,seed", [((4, 4, 6), 1), ((6, 6, 6), 2), ((4, 6, 4), 5)])
def test_random_vs_lapack(orc, shape, seed):
    w = wk.random_small(*shape, seed=seed, n_vortices=2)
    pins.check_vs_lapack(orc.build, orc.heev, w)
    H = orc.build(w)
    ev, Z = orc.heev(H)
    rho = np.max(np.abs(ev))
    assert np.max(np.linalg.norm(H @ Z - Z * ev, axis=0)) / rho < 1e-13
    assert orc.orthogonality(Z) < 1e-12
    # spectral projectors of well-separated eigenvalues agree with LAPACK's vectors
    ref_w, ref_Z = np.linalg.eigh(H)
    gaps = np.minimum(np.abs(np.diff(ev, prepend=-np.inf)), np.abs(np.diff(ev, append=np.inf)))
    iso = np.nonzero(gaps > 1e-6 * rho)[0]
    ov = np.abs(np.sum(Z[:, iso].conj() * ref_Z[:, iso], axis=0))
    assert np.min(ov) > 1 - 1e-9


def test_particle_hole_pairing_and_sums(orc):
    """(u, v) at E implies (-v^*, u^*) at -E; sum E = tr H = 0; sum E^2 = ||H||_F^2."""
    w = wk.random_small(4, 4, 6, seed=7, n_vortices=2)
    H = orc.build(w)
    ev, Z = orc.heev(H)
    rho = np.max(np.abs(ev))
    assert np.max(np.abs(ev + ev[::-1])) / rho < 1e-13
    V = w.V
    Zp = np.concatenate([-Z[V:].conj(), Z[:V].conj()])
    assert np.max(np.linalg.norm(H @ Zp + Zp * ev, axis=0)) / rho < 1e-13
    assert abs(ev.sum()) / rho < 1e-11
    f2 = pins.frobenius2_closed_form(w)
    assert abs(np.sum(ev ** 2) - f2) / f2 < 1e-13


def test_tridiagonal_reduction_inertia(orc):
    """The real tridiagonal the oracle reduces H to has the same inertia as H at
    any shift (Sturm count vs number of LAPACK eigenvalues below the shift)."""
    w = wk.random_small(4, 4, 4, seed=11, n_vortices=1)
    H = orc.build(w)
    d, e, tau, _ = orc.tridiag(H)
    er, D = orc.phase(e)
    assert np.all(er >= 0)
    ref = np.linalg.eigvalsh(H)
    rng = np.random.default_rng(0)
    for sigma in rng.uniform(ref[0] - 1, ref[-1] + 1, 25):
        assert orc.sturm_count(d, er, sigma) == int(np.sum(ref < sigma))


def test_tridiagonal_qr_vs_scipy(orc):
    rng = np.random.default_rng(4)
    for n in (1, 2, 3, 17, 200):
        d = rng.standard_normal(n)
        e = rng.standard_normal(max(n - 1, 0))
        if n > 5:
            e[n // 3] = 0.0                      # a split
            d[-3:] = d[-4]                       # repeated diagonal entries
        ev, Q = orc.tqr(d, e, vectors=True)
        ref = scipy.linalg.eigh_tridiagonal(d, e, eigvals_only=True) if n > 1 else d
        assert np.max(np.abs(np.sort(ev) - ref)) < 1e-13 * max(1.0, np.max(np.abs(ref)))
        T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
        assert np.max(np.abs(T @ Q - Q * ev)) < 1e-13 * max(1.0, np.max(np.abs(ref)))
        assert np.max(np.abs(Q.T @ Q - np.eye(n))) < 1e-13


def test_apply_matches_dense_and_fft(orc):
    w = wk.random_small(4, 6, 4, seed=2, n_vortices=1)
    H = orc.build(w)
    X = wk.unit_vectors(w.N, 5, seed=3)
    Y = orc.apply(w, X)
    assert np.max(np.abs(Y - H @ X)) < 1e-13
    # independent route: kinetic term through numpy FFTs on the 3-D grid
    shape = (w.nx, w.ny, w.nz)
    ks = []
    for n in shape:
        k = 2 * np.pi * np.fft.fftfreq(n)
        k[np.isclose(k, np.pi)] = -np.pi
        ks.append(k)
    kx, ky, kz = np.meshgrid(*ks, indexing="ij")
    k2h = 0.5 * (kx ** 2 + ky ** 2 + kz ** 2)
    V = w.V
    for c in range(X.shape[1]):
        u = X[:V, c].reshape(shape)
        v = X[V:, c].reshape(shape)
        Tu = np.fft.ifftn(k2h * np.fft.fftn(u)).ravel()
        Tv = np.fft.ifftn(k2h * np.fft.fftn(v)).ravel()
        yu = Tu + (w.U - w.mu) * u.ravel() + w.Delta * v.ravel()
        yv = w.Delta.conj() * u.ravel() - (Tv + (w.U - w.mu) * v.ravel())
        assert np.max(np.abs(Y[:V, c] - yu)) < 1e-12
        assert np.max(np.abs(Y[V:, c] - yv)) < 1e-12


def test_uniform_densities_closed_form(orc):
    """n = (2/V) sum v_k^2, nu = (1/V) sum Delta/(2E_k) over 0 < E_k < E_c."""
    pins.check_uniform_densities(orc.build, orc.heev, orc.densities, 4, 4, 6)


@pytest.mark.parametrize("T", [0.05, 0.2])
def test_uniform_densities_finite_temperature_closed_form(orc, T):
    """The BCS sums with tanh(E/2T) weights (the Fermi weights of Eq. (n))."""
    pins.check_uniform_densities(orc.build, orc.heev, orc.densities, 4, 4, 6, T=T)


def test_finite_temperature_densities_reduce(orc):
    """At small T the Fermi-weighted densities approach the T=0 ones (gap 0.2)."""
    w = wk.random_small(4, 4, 4, seed=5, n_vortices=0)
    ev, Z = orc.heev(orc.build(w))
    n0, nu0 = orc.densities(ev, Z, w.V, T=0.0)
    n1, nu1 = orc.densities(ev, Z, w.V, T=1e-4)
    assert np.max(np.abs(n1 - n0)) < 1e-12 and np.max(np.abs(nu1 - nu0)) < 1e-12


def test_pairing_field_phase_follows_delta(orc):
    w = wk.random_small(6, 6, 4, seed=9, n_vortices=1, amplitude=0.4)
    pins.check_pairing_phase(orc.build, orc.heev, orc.densities, w)


def test_scf_uniform_fixed_point(orc):
    """With g from the lattice gap equation, the uniform (U0, Delta0) state is a
    fixed point of the self-consistent update."""
    pins.check_scf_fixed_point(orc.scf_step, orc.gap_coupling, 4, 4, 4)


def test_scf_update_keeps_vortex_phase(orc):
    w = wk.random_small(6, 6, 4, seed=9, n_vortices=1, amplitude=0.4)
    g, _ = orc.gap_coupling(6, 6, 4, w.mu, 0.4)
    pins.check_scf_phase(orc.scf_step, w, g)


def test_cutoff_count_matches_paper_estimate(orc):
    """The number of states with 0 < E < E_c = pi^2/2 is of order 0.5 V
    (paper's estimate 4/3 pi k_max^3 / (dk)^3 = (pi/6) V, stored in golden)."""
    import json, os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
    w = wk.c1_uniform()
    ev = orc.heev(orc.build(w), vectors=False)
    cnt = np.sum((ev > 0) & (ev < g["E_c"]))
    assert abs(cnt / w.V - g["qpwf_per_site_estimate"]) < 0.1


def test_kz_block_decomposition(orc):
    """A z-invariant system splits into kz blocks H_kz = H_perp(mu - kz^2/2):
    the union of the block spectra is the 3-D spectrum (and a size-1 grid
    dimension carries only k = 0)."""
    import workloads as wk
    nx, ny, nz = 4, 4, 6
    D2 = wk.vortex_pairing(nx, ny, 1, 0.3, [(0.4, 0.1)], [1]).reshape(-1)
    U2 = (-0.4 + wk.smooth_field((nx, ny), 2.0, 3, 0.05)).reshape(-1)
    w3 = wk.Workload("zinv", nx, ny, nz, 0.5, np.repeat(U2, nz), np.repeat(D2, nz), {})
    ew = orc.heev(orc.build(w3), vectors=False)
    parts = []
    for m in range(-nz // 2, nz // 2):
        kz = 2 * np.pi * m / nz
        wb = wk.Workload("blk", nx, ny, 1, 0.5 - 0.5 * kz * kz, U2, D2, {})
        parts.append(orc.heev(orc.build(wb), vectors=False))
    union = np.sort(np.concatenate(parts))
    assert np.max(np.abs(union - ew)) <= 1e-12 * np.max(np.abs(ew))
    T1, _ = orc.kinetic_1d(1)
    assert T1[0, 0] == 0.0


def test_uniform_tube_kz_blocks_closed_form(orc):
    """Uniform tube (U = 0, constant Delta0): the block of wave number kz, built on the
    (nx, ny, 1) grid with mu - kz^2/2, has E = +-sqrt((k_perp^2/2 + kz^2/2 - mu)^2 + Delta0^2);
    the blocks of +kz and -kz coincide."""
    nx, ny, nz, mu, D0 = 6, 4, 8, 0.5, 0.3
    kp = pins.lattice_k2half(nx, ny, 1)
    spectra = {}
    for m in range(-nz // 2, nz // 2):
        kz = 2 * np.pi * m / nz
        wb = wk.uniform(nx, ny, 1, mu - 0.5 * kz * kz, 0.0, D0)
        ev = np.sort(orc.heev(orc.build(wb), vectors=False))
        E = np.sqrt((kp + 0.5 * kz * kz - mu) ** 2 + D0 ** 2)
        ref = np.sort(np.concatenate([-E, E]))
        assert np.max(np.abs(ev - ref)) < 1e-13 * np.max(np.abs(ref))
        spectra[m] = ev
    for m in range(1, nz // 2):
        assert np.max(np.abs(spectra[m] - spectra[-m])) < 1e-13


@pytest.mark.parametrize("T", [0.0, 0.1])
def test_uniform_kinetic_density_closed_form(orc, T):
    pins.check_uniform_tau(orc.build, orc.heev, orc.kinetic_current_densities, 4, 4, 6, T=T)


def test_kinetic_density_integrates_to_twice_the_kinetic_energy(orc):
    """sum_r |grad f|^2 = 2 <f|T|f> with T the kinetic block of the built H (Parseval), so
    sum_r tau = 4 sum_n (<v_n|T|v_n> f_T(-E_n) + <u_n|T|u_n> f_T(E_n))."""
    w = wk.random_small(6, 4, 4, seed=4, n_vortices=1, amplitude=0.4)
    H = orc.build(w)
    ev, Z = orc.heev(H)
    V = w.V
    Tk = H[:V, :V] - np.diag(w.U - w.mu)
    for T in (0.0, 0.15):
        tau, _ = orc.kinetic_current_densities(ev, Z, (w.nx, w.ny, w.nz), T=T)
        sel = np.nonzero((ev > 0) & (ev < np.pi ** 2 / 2))[0]
        u, v = Z[:V, sel], Z[V:, sel]
        eu = np.real(np.einsum("ij,ik,kj->j", u.conj(), Tk, u))
        evv = np.real(np.einsum("ij,ik,kj->j", v.conj(), Tk, v))
        ref = 4.0 * (evv @ orc.fermi(-ev[sel], T) + eu @ orc.fermi(ev[sel], T))
        assert abs(tau.sum() - ref) < 1e-12 * ref


def test_real_hamiltonian_carries_no_current(orc):
    w = wk.random_small(6, 4, 4, seed=2, n_vortices=0)
    w.Delta = np.abs(w.Delta) + 0j
    ev, Z = orc.heev(orc.build(w))
    _, j = orc.kinetic_current_densities(ev, Z, (w.nx, w.ny, w.nz), T=0.05)
    assert np.max(np.abs(j)) < 1e-13


@pytest.mark.parametrize("sign", [1, -1])
def test_pairing_boost_carries_the_galilean_current(orc, sign):
    pins.check_boost_current(orc.build, orc.heev, orc.densities, orc.kinetic_current_densities, sign)


@pytest.mark.parametrize("charge", [1, -1])
def test_vortex_current_circulates_with_its_winding(orc, charge):
    pins.check_vortex_circulation(orc.build, orc.heev, orc.kinetic_current_densities, charge)
