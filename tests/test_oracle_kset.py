"""The lattice k set of the oracle's kinetic operator (paper, "Numerical setup and implementation":
the spectral k^2/2 on k = 2 pi m / n) for every dimension length: even n gives m = -n/2 .. n/2-1,
odd n the symmetric -(n-1)/2 .. (n-1)/2, and a size-1 dimension k = 0 only.  The eigenvalues of the
oracle's DFT-sum kinetic matrix and its kinetic-energy list must be k^2/2 over exactly that set."""
import math

import numpy as np
import pytest

import oracle


def k2half(n):
    m = np.arange(-(n // 2), n - n // 2)
    return np.sort(0.5 * (2 * math.pi * m / n) ** 2)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8])
def test_kinetic_matrix_spectrum_is_k2_over_the_lattice_set(n):
    T, im = oracle.kinetic_1d(n)
    assert im < 1e-12
    assert np.allclose(np.sort(np.linalg.eigvalsh(T)), k2half(n), atol=1e-12)


@pytest.mark.parametrize("shape", [(1, 4, 6), (3, 4, 2), (5, 1, 1), (4, 4, 4)])
def test_kinetic_energies_match_the_kinetic_matrix(shape):
    nx, ny, nz = shape
    Tx, _ = oracle.kinetic_1d(nx)
    Ty, _ = oracle.kinetic_1d(ny)
    Tz, _ = oracle.kinetic_1d(nz)
    K = (np.kron(np.kron(Tx, np.eye(ny)), np.eye(nz)) + np.kron(np.kron(np.eye(nx), Ty), np.eye(nz))
         + np.kron(np.kron(np.eye(nx), np.eye(ny)), Tz))
    assert np.allclose(np.sort(np.linalg.eigvalsh(K)), np.sort(oracle.kinetic_energies(nx, ny, nz)), atol=1e-11)
