"""Checks that pin the oracle to facts fixed by the paper and by mathematics.

Each check takes the operator/eigensolver callables as arguments so that the
mutation tests can feed it a deliberately broken variant and confirm that the
check fails.  Nothing here calls the CUDA library.
"""
import numpy as np

import workloads as wk


def closed_form_kinetic_column(n):
    """t(d) for the spectral kinetic matrix on n points (d = 0..n-1):
    t(0) = pi^2 (n^2 + 2) / (6 n^2), t(d) = (-1)^d pi^2 / (n^2 sin^2(pi d / n))."""
    d = np.arange(n)
    out = np.empty(n)
    out[0] = np.pi ** 2 * (n * n + 2) / (6.0 * n * n)
    dd = d[1:]
    out[1:] = (-1.0) ** dd * np.pi ** 2 / (n * n * np.sin(np.pi * dd / n) ** 2)
    return out


def lattice_k2half(nx, ny, nz):
    # k = 2 pi m / n, m = -n/2 .. n/2-1 for even n; a size-1 dimension has k = 0 only
    ks = [2 * np.pi * np.arange(-(n // 2), n - n // 2) / n for n in (nx, ny, nz)]
    kx, ky, kz = np.meshgrid(*ks, indexing="ij")
    return (0.5 * (kx ** 2 + ky ** 2 + kz ** 2)).ravel()


def uniform_spectrum(nx, ny, nz, mu, U0, D0):
    """E = +-sqrt((k^2/2 - mu + U0)^2 + |Delta0|^2) over the spectral k grid."""
    xi = lattice_k2half(nx, ny, nz) - mu + U0
    E = np.sqrt(xi * xi + abs(D0) ** 2)
    return np.sort(np.concatenate([-E, E]))


def frobenius2_closed_form(w):
    """||H||_F^2 = 2 ||h||_F^2 + 2 sum |Delta|^2, with ||h||_F^2 from Parseval:
    sum_k (k^2/2)^2 + 2 tr(T) mean-shift term + sum c^2, c = U - mu."""
    V = w.V
    e = lattice_k2half(w.nx, w.ny, w.nz)
    diagT = e.sum() / V                      # every diagonal entry of T equals tr(T)/V
    c = w.U - w.mu
    h2 = np.sum(e * e) + 2.0 * diagT * c.sum() + np.sum(c * c)
    return 2.0 * h2 + 2.0 * np.sum(np.abs(w.Delta) ** 2)


def check_uniform(build, heev, nx, ny, nz, mu=0.5, D0=0.2, tol=1e-12):
    w = wk.uniform(nx, ny, nz, mu, 0.0, D0)
    ev = heev(build(w), vectors=False)
    ref = uniform_spectrum(nx, ny, nz, mu, 0.0, D0)
    rho = np.max(np.abs(ref))
    err = np.max(np.abs(np.sort(ev) - ref)) / rho
    assert err <= tol, f"uniform spectrum error {err:.3e}"
    return err


def check_vs_lapack(build, heev, w, tol=1e-12):
    H = build(w)
    ev = heev(H, vectors=False)
    ref = np.linalg.eigvalsh(H)
    rho = np.max(np.abs(ref))
    err = np.max(np.abs(np.sort(ev) - ref)) / rho
    assert err <= tol, f"eigenvalue error vs LAPACK {err:.3e}"
    return err


def check_frobenius_and_trace(build, w, tol=1e-12):
    H = build(w)
    f2 = np.sum(np.abs(H) ** 2)
    ref = frobenius2_closed_form(w)
    assert abs(f2 - ref) <= tol * ref, f"||H||_F^2 {f2} vs closed form {ref}"
    tr = np.trace(H)
    assert abs(tr) <= tol * np.sqrt(ref), f"trace {tr}"


def check_pairing_phase(build, heev, densities, w):
    """nu must wind like Delta: Re(nu conj(Delta)) > 0 wherever |Delta| is not small
    (upper-right block Delta, lower-left Delta^*, nu = sum u v^*)."""
    H = build(w)
    ev, Z = heev(H, vectors=True)
    n, nu = densities(ev, Z, w.V)
    mask = np.abs(w.Delta) > 0.5 * np.max(np.abs(w.Delta))
    c = np.real(nu[mask] * np.conj(w.Delta[mask])) / (np.abs(nu[mask]) * np.abs(w.Delta[mask]))
    assert np.min(c) > 0.9, f"nu does not follow the phase of Delta (min cos {np.min(c):.3f})"


def check_uniform_densities(build, heev, densities, nx, ny, nz, mu=0.5, D0=0.2, T=0.0, tol=1e-13):
    """Uniform state, BCS occupations: with xi = k^2/2 - mu, E = sqrt(xi^2 + D0^2) and
    u^2, v^2 = (1 +- xi/E)/2 per plane wave, the Fermi-weighted sums over 0 < E < E_c are
    n = (1/V) sum [1 - (xi/E) tanh(E/2T)] and nu = (1/V) sum D0 tanh(E/2T) / (2E)
    (tanh -> 1 at T = 0).  Degenerate shells enter whole, so the split of a shell's
    eigenvectors does not matter."""
    w = wk.uniform(nx, ny, nz, mu, 0.0, D0)
    ev, Z = heev(build(w), vectors=True)
    n, nu = densities(ev, Z, w.V, T=T)
    xi = lattice_k2half(nx, ny, nz) - mu
    E = np.sqrt(xi ** 2 + D0 ** 2)
    sel = E < np.pi ** 2 / 2
    th = np.ones(int(sel.sum())) if T == 0.0 else np.tanh(E[sel] / (2.0 * T))
    n0 = np.sum(1.0 - xi[sel] / E[sel] * th) / w.V
    nu0 = np.sum(D0 * th / (2.0 * E[sel])) / w.V
    err_n, err_nu = np.max(np.abs(n - n0)), np.max(np.abs(nu - nu0))
    assert err_n < tol and err_nu < tol, f"uniform densities: n err {err_n:.3e}, nu err {err_nu:.3e}"


def check_scf_fixed_point(scf_step, gap_coupling, nx, ny, nz, mu=0.5, D0=0.25, tol=1e-12):
    """With g and U0 from the gap equation of the uniform state, (U0, D0) is a fixed point of
    the self-consistent update at any mixing."""
    g, U0 = gap_coupling(nx, ny, nz, mu, D0)
    assert g > 0 and U0 < 0
    w = wk.uniform(nx, ny, nz, mu, U0, D0)
    U1, D1, _, _ = scf_step(w, g, alpha=1.0)
    err = max(np.max(np.abs(U1 - U0)), np.max(np.abs(D1 - D0)))
    assert err < tol, f"uniform fixed point moved by {err:.3e}"


def check_scf_phase(scf_step, w, g):
    """An attractive coupling (g > 0) keeps the phase of the pairing field: after one full
    update the new Delta has Re(Delta_new conj(Delta_old)) > 0 wherever |Delta_old| is not
    small, so a vortex keeps its winding."""
    _, D1, _, _ = scf_step(w, g, alpha=1.0)
    mask = np.abs(w.Delta) > 0.5 * np.max(np.abs(w.Delta))
    c = np.real(D1[mask] * np.conj(w.Delta[mask])) / (np.abs(D1[mask]) * np.abs(w.Delta[mask]))
    assert np.min(c) > 0.9, f"the update does not keep the phase of Delta (min cos {np.min(c):.3f})"


def check_uniform_tau(build, heev, kcd, nx, ny, nz, mu=0.5, D0=0.3, T=0.0, tol=1e-12):
    """Uniform state: each plane-wave pair adds k^2/V times its occupation, so
    tau = (1/V) sum k^2 [1 - (xi/E) tanh(E/2T)] over 0 < E < E_c (k^2 = 2 x the kinetic
    energy of the k set), and there is no current."""
    w = wk.uniform(nx, ny, nz, mu, 0.0, D0)
    ev, Z = heev(build(w), vectors=True)
    tau, j = kcd(ev, Z, (nx, ny, nz), T=T)
    k2 = 2.0 * lattice_k2half(nx, ny, nz)
    xi = 0.5 * k2 - mu
    E = np.sqrt(xi ** 2 + D0 ** 2)
    sel = E < np.pi ** 2 / 2
    th = np.ones(int(sel.sum())) if T == 0.0 else np.tanh(E[sel] / (2.0 * T))
    tau0 = np.sum(k2[sel] * (1.0 - xi[sel] / E[sel] * th)) / w.V
    assert np.max(np.abs(tau - tau0)) < tol * tau0, f"uniform tau {tau[0]} vs {tau0}"
    assert np.max(np.abs(j)) < 1e-13, f"uniform state carries a current {np.max(np.abs(j)):.2e}"


def check_boost_current(build, heev, densities, kcd, sign=1, tol=0.02):
    """Pairing field Delta0 e^{i q x} on a 24x4x4 lattice with q = 4 pi / 24 (small against the
    zone): the pairs move with momentum q, so j = n q / 2 along x (Galilean boost, up to the
    cutoff window), uniform, with no y or z component."""
    shape, mu, D0 = (24, 4, 4), 0.5, 0.3
    q = sign * 4 * np.pi / shape[0]
    x, _, _ = wk.coords(*shape)
    V = int(np.prod(shape))
    w = wk.Workload("boost", *shape, mu, np.zeros(V), D0 * np.exp(1j * q * (x + shape[0] / 2)), {})
    ev, Z = heev(build(w), vectors=True)
    n, _ = densities(ev, Z, V)
    _, j = kcd(ev, Z, shape)
    ratio = np.mean(j[0]) / (np.mean(n) * q / 2)
    assert abs(ratio - 1.0) < tol, f"j_x / (n q/2) = {ratio:.4f}"
    assert np.max(j[0]) - np.min(j[0]) < 1e-12 and np.max(np.abs(j[1:])) < 1e-13


def check_vortex_circulation(build, heev, kcd, charge):
    """A vortex of winding +-1 on the z axis: around the core the current circulates with the
    sense of the winding (j . phi_hat has the sign of the charge)."""
    shape = (8, 8, 2)
    D = wk.vortex_pairing(*shape, 0.4, [(0.0, 0.0)], [charge])
    V = int(np.prod(shape))
    w = wk.Workload("vortex", *shape, 0.5, np.zeros(V), D, {})
    ev, Z = heev(build(w), vectors=True)
    _, j = kcd(ev, Z, shape)
    x, y, _ = wk.coords(*shape)
    rho = np.hypot(x, y)
    ring = (rho > 0.5) & (rho < 2.5)
    jphi = (-y[ring] * j[0][ring] + x[ring] * j[1][ring]) / rho[ring]
    assert np.all(charge * jphi > 0), f"circulation sense {np.sign(jphi)} for charge {charge}"
