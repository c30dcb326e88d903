"""FP64 CPU oracle for the static BdG eigenproblem -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The CUDA
library never calls it and shares no code with it; the only thing both sides
share is the seeded input generator in ``workloads``.

What it computes (each function names the passage it follows):

* ``kinetic_1d``  -- the spectral kinetic matrix F^-1 (k^2/2) F, k = 2 pi m/n,
  m = -n/2..n/2-1 (paper, "Numerical setup and implementation").
* ``build``       -- the dense quasiparticle Hamiltonian of Eq. (stHpsi).
* ``apply``       -- the same operator applied matrix-free.
* ``heev``        -- all eigenpairs: unblocked Householder tridiagonalisation,
  implicit symmetric QR with rotations accumulated, back-transformation
  (the 1-stage reduction / tridiagonal solve / back-transformation sequence the
  paper describes for its eigensolver, "Performance of the Matrix
  Diagonalization Algorithm").
* ``densities``   -- n(r) and nu(r) of Eq. (densities2) with the Fermi function
  f_T and the window 0 < E_n < E_c.
* ``kinetic_current_densities`` -- tau(r) and j(r) of the same equation, with
  the spectral gradient F^-1 (i k) F on the lattice's k set.
* ``gap_coupling`` / ``scf_step`` -- one self-consistent update with the stated
  substitute functional (contact coupling with Hartree term: Delta = g nu,
  U = -g n / 2, g fixed by the lattice gap equation of the uniform state).
  Parity with the paper's SLDA functional is unpinned: its B and C functions
  are not printed in the paper.

The compiled part lives in ``bdg_oracle.c`` and is built by ``build_lib()``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liborc.so")
_SRC = os.path.join(_HERE, "bdg_oracle.c")
_lib = None


def build_lib(force: bool = False) -> str:
    """Compile bdg_oracle.c into oracle/liborc.so (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", _LIB_PATH, _SRC, "-lm"])
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build_lib()
        L = C.CDLL(_LIB_PATH)
        P = C.c_void_p
        i64 = C.c_int64
        L.orc_kinetic_1d.argtypes = [C.c_int, P, P]
        L.orc_build.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, P, P, P, i64]
        L.orc_apply.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, P, P, i64, P, i64, P, i64, C.c_int]
        L.orc_tridiag.argtypes = [i64, P, i64, P, P, P, C.c_int]
        L.orc_phase.argtypes = [i64, P, P, P]
        L.orc_tqr.argtypes = [i64, P, P, P, i64, C.c_int]
        L.orc_tqr.restype = C.c_int
        L.orc_backtransform.argtypes = [i64, P, i64, P, i64, P, i64, C.c_int]
        L.orc_heev.argtypes = [i64, P, i64, P, P, i64, C.c_int]
        L.orc_heev.restype = C.c_int
        L.orc_sturm_count.argtypes = [i64, P, P, C.c_double]
        L.orc_sturm_count.restype = i64
        L.orc_max_threads.restype = C.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def max_threads() -> int:
    return int(lib().orc_max_threads())


# ----------------------------------------------------------------------------
# operator
# ----------------------------------------------------------------------------
def kinetic_1d(n: int):
    """(T, max |Im|): the n x n kinetic matrix from the inverse-DFT sum."""
    T = np.zeros((n, n), dtype=np.float64, order="F")
    im = np.zeros(1)
    lib().orc_kinetic_1d(n, _p(T), _p(im))
    return T, float(im[0])


def build(w) -> np.ndarray:
    """Dense H (N x N complex128, Fortran order) for a workloads.Workload."""
    N = w.N
    H = np.zeros((N, N), dtype=np.complex128, order="F")
    U = np.ascontiguousarray(w.U, dtype=np.float64)
    D = np.ascontiguousarray(w.Delta, dtype=np.complex128)
    lib().orc_build(w.nx, w.ny, w.nz, float(w.mu), _p(U), _p(D), _p(H), N)
    return H


def apply(w, X: np.ndarray, threads: int = 0) -> np.ndarray:
    """Matrix-free Y = H X (X: N x k, any layout; returns Fortran-order N x k)."""
    X = np.asfortranarray(X, dtype=np.complex128)
    if X.ndim == 1:
        X = X.reshape(-1, 1, order="F")
    Y = np.zeros_like(X, order="F")
    U = np.ascontiguousarray(w.U, dtype=np.float64)
    D = np.ascontiguousarray(w.Delta, dtype=np.complex128)
    lib().orc_apply(w.nx, w.ny, w.nz, float(w.mu), _p(U), _p(D), X.shape[1], _p(X), X.shape[0],
                    _p(Y), Y.shape[0], int(threads))
    return Y


# ----------------------------------------------------------------------------
# eigensolver
# ----------------------------------------------------------------------------
def tridiag(H: np.ndarray, threads: int = 0):
    """Householder tridiagonalisation: (d, e_complex, tau, A_with_reflectors)."""
    A = np.array(H, dtype=np.complex128, order="F", copy=True)
    n = A.shape[0]
    d = np.zeros(n)
    e = np.zeros(max(n - 1, 1), dtype=np.complex128)
    tau = np.zeros(max(n - 1, 1))
    lib().orc_tridiag(n, _p(A), n, _p(d), _p(e), _p(tau), int(threads))
    return d, e[: n - 1], tau[: n - 1], A


def phase(e: np.ndarray):
    """(|e|, D) with D_0 = 1, D_{k+1} = D_k e_k/|e_k| (real tridiagonal = D^H T D)."""
    n = e.shape[0] + 1
    er = np.zeros(max(n - 1, 1))
    D = np.zeros(n, dtype=np.complex128)
    e = np.ascontiguousarray(e, dtype=np.complex128)
    lib().orc_phase(n, _p(e), _p(er), _p(D))
    return er[: n - 1], D


def tqr(d: np.ndarray, e: np.ndarray, vectors: bool = False, threads: int = 0):
    """Eigenvalues (unsorted) and optionally eigenvectors of a real tridiagonal."""
    d = np.array(d, dtype=np.float64, copy=True)
    n = d.shape[0]
    e = np.ascontiguousarray(e, dtype=np.float64)
    Q = None
    if vectors:
        Q = np.asfortranarray(np.eye(n))
    st = lib().orc_tqr(n, _p(d), _p(e), _p(Q) if vectors else None, n, int(threads))
    if st != 0:
        raise RuntimeError("oracle tridiagonal QR did not converge")
    return (d, Q) if vectors else d


def sturm_count(d: np.ndarray, e: np.ndarray, sigma: float) -> int:
    d = np.ascontiguousarray(d, dtype=np.float64)
    e = np.ascontiguousarray(e, dtype=np.float64)
    return int(lib().orc_sturm_count(d.shape[0], _p(d), _p(e), float(sigma)))


def heev(H: np.ndarray, vectors: bool = True, threads: int = 0):
    """All eigenpairs of the Hermitian H (not modified). Returns w or (w, Z)."""
    A = np.array(H, dtype=np.complex128, order="F", copy=True)
    n = A.shape[0]
    w = np.zeros(n)
    Z = np.zeros((n, n), dtype=np.complex128, order="F") if vectors else None
    st = lib().orc_heev(n, _p(A), n, _p(w), _p(Z) if vectors else None, n, int(threads))
    if st != 0:
        raise RuntimeError("oracle eigensolver did not converge")
    return (w, Z) if vectors else w


# ----------------------------------------------------------------------------
# densities and the self-consistent update
# ----------------------------------------------------------------------------
def fermi(E: np.ndarray, T: float) -> np.ndarray:
    """f_T(E) = 1/(1+exp(E/T)); at T = 0 the step with f(0) = 1/2."""
    E = np.asarray(E, dtype=np.float64)
    if T == 0.0:
        return np.where(E < 0, 1.0, np.where(E > 0, 0.0, 0.5))
    return 0.5 * (1.0 - np.tanh(E / (2.0 * T)))


def densities(w: np.ndarray, Z: np.ndarray, V: int, T: float = 0.0, Ec: float = np.pi ** 2 / 2):
    """n(r), nu(r) of Eq. (densities2) over the states with 0 < E_n < E_c."""
    sel = np.nonzero((w > 0.0) & (w < Ec))[0]
    E = w[sel]
    u = Z[:V, sel]
    v = Z[V:, sel]
    fp, fm = fermi(E, T), fermi(-E, T)
    n = 2.0 * ((np.abs(v) ** 2) @ fm + (np.abs(u) ** 2) @ fp)
    nu = (u * np.conj(v)) @ (fm - fp)
    return n, nu


def spectral_gradient(F: np.ndarray, shape, keep_nyquist: bool):
    """Gradient components of site fields given by their DFT F (axes 0..2 of shape + (columns,)):
    d_a f = F^-1 (i k_a) F with k_a = 2 pi m / n_a, m = -n_a/2 .. n_a/2-1 (the kinetic operator's
    k set; paper, "Numerical setup and implementation").  keep_nyquist=False gives the m = -n_a/2 mode the derivative 0 (the mean of its
    +-pi images)."""
    out = []
    for a, n in enumerate(shape):
        k = 2.0 * np.pi * np.fft.fftfreq(n)            # FFT order; index n/2 holds m = -n/2
        if not keep_nyquist:
            k[n // 2] = 0.0
        sh = [1] * F.ndim
        sh[a] = n
        out.append(np.fft.ifftn(1j * k.reshape(sh) * F, axes=(0, 1, 2)))
    return out


def kinetic_current_densities(w: np.ndarray, Z: np.ndarray, shape, T: float = 0.0,
                              Ec: float = np.pi ** 2 / 2):
    """tau(r) and j(r) = (j_x, j_y, j_z) of Eq. (densities2) over the states with 0 < E_n < E_c:
      tau = 2 sum (|grad v|^2 f_T(-E) + |grad u|^2 f_T(E)),
      j   = 2 sum Im(v grad v^* f_T(-E) - u grad u^* f_T(E)).
    tau takes the k set as written, so that sum_r tau is twice the kinetic energy of the
    build's kinetic operator; j gives the Nyquist mode the derivative 0, so that a real
    (time-reversal invariant) state carries no current.  Returns (tau (V,), j (3, V))."""
    shape = tuple(int(x) for x in shape)
    V = int(np.prod(shape))
    sel = np.nonzero((w > 0.0) & (w < Ec))[0]
    E = w[sel]
    fp, fm = fermi(E, T), fermi(-E, T)
    u = Z[:V, sel].reshape(shape + (len(sel),))
    v = Z[V:, sel].reshape(shape + (len(sel),))
    Fu, Fv = np.fft.fftn(u, axes=(0, 1, 2)), np.fft.fftn(v, axes=(0, 1, 2))
    tau = np.zeros(shape)
    for gu, gv in zip(spectral_gradient(Fu, shape, True), spectral_gradient(Fv, shape, True)):
        tau += 2.0 * (np.abs(gv) ** 2 @ fm + np.abs(gu) ** 2 @ fp)
    j = [2.0 * np.imag((v * np.conj(gv)) @ fm - (u * np.conj(gu)) @ fp)
         for gu, gv in zip(spectral_gradient(Fu, shape, False), spectral_gradient(Fv, shape, False))]
    return tau.reshape(-1), np.stack([c.reshape(-1) for c in j])


def kinetic_energies(nx: int, ny: int, nz: int) -> np.ndarray:
    """k^2/2 on the spectral grid in site order (eigenvalues of the kinetic operator)."""
    # m = -floor(n/2) .. n - floor(n/2) - 1: for even n -n/2 .. n/2-1; a size-1 dimension has k = 0 only
    ks = [2 * np.pi * np.arange(-(n // 2), n - n // 2) / n for n in (nx, ny, nz)]
    kx, ky, kz = np.meshgrid(*ks, indexing="ij")
    return (0.5 * (kx ** 2 + ky ** 2 + kz ** 2)).ravel()


def uniform_sums(nx, ny, nz, mu, U0, Delta0, Ec=np.pi ** 2 / 2):
    """(n0, nu0/Delta0 * Delta0, E_k) of the uniform state summed over 0 < E_k < E_c."""
    V = nx * ny * nz
    eps = kinetic_energies(nx, ny, nz)
    xi = eps - mu + U0
    E = np.sqrt(xi * xi + abs(Delta0) ** 2)
    sel = (E > 0) & (E < Ec)
    n0 = (2.0 / V) * np.sum(0.5 * (1.0 - xi[sel] / E[sel]))
    nu0 = (1.0 / V) * np.sum(Delta0 / (2.0 * E[sel]))
    return n0, nu0, E


def gap_coupling(nx, ny, nz, mu, Delta0, Ec=np.pi ** 2 / 2, iters=200):
    """Coupling g > 0 and Hartree shift U0 that make the uniform state with gap
    Delta0 self-consistent: Delta0 = g nu0 and U0 = -g n0/2."""
    g = 1.0
    U0 = 0.0
    for _ in range(iters):
        n0, nu0, _ = uniform_sums(nx, ny, nz, mu, U0, Delta0, Ec)
        g_new = Delta0 / nu0
        U_new = -g_new * n0 / 2.0
        if abs(g_new - g) < 1e-15 * abs(g) and abs(U_new - U0) < 1e-15:
            g, U0 = g_new, U_new
            break
        g, U0 = g_new, U_new
    return float(g), float(U0)


def scf_step(w, g: float, alpha: float = 0.3, phase=None, T: float = 0.0, Ec: float = np.pi ** 2 / 2,
             threads: int = 0):
    """One self-consistent step: H(U, Delta) -> eigenpairs -> (n, nu) -> mixed update.

    Returns (U_new, Delta_new, n, nu, max|dn| placeholder None).  With a fixed
    phase field `phase` (unit complex), Delta_out = g Re(nu e^{-i theta}) e^{i theta}.
    """
    H = build(w)
    ev, Z = heev(H, vectors=True, threads=threads)
    n, nu = densities(ev, Z, w.V, T, Ec)
    U_out = -g * n / 2.0
    if phase is None:
        D_out = g * nu
    else:
        D_out = g * np.real(nu * np.conj(phase)) * phase
    U_new = (1.0 - alpha) * w.U + alpha * U_out
    D_new = (1.0 - alpha) * w.Delta + alpha * D_out
    return U_new, D_new, n, nu


# ----------------------------------------------------------------------------
# accuracy measures (the error norms every result is reported with)
# ----------------------------------------------------------------------------
def residuals(wl, w: np.ndarray, Z: np.ndarray, cols=None, threads: int = 0) -> np.ndarray:
    """||H z_i - w_i z_i||_2 for the selected columns (matrix-free H)."""
    if cols is None:
        cols = np.arange(Z.shape[1])
    Zs = np.asfortranarray(Z[:, cols])
    Y = apply(wl, Zs, threads)
    return np.linalg.norm(Y - Zs * w[cols][None, :], axis=0)


def orthogonality(Z: np.ndarray) -> float:
    """max |Z^H Z - I|."""
    G = Z.conj().T @ Z
    return float(np.max(np.abs(G - np.eye(G.shape[0]))))
