"""Dense-matrix and Fourier constructions of the periodic operators, written for the
tests independently of the oracle (numpy only).  Used to pin the oracle."""
import numpy as np


def shape_of(n):
    return tuple(reversed(n))  # numpy shape, x fastest


def dense_A(n):
    """Dense A (N x N): sum_a n_a^2 (2 I - S_a - S_a^T), S_a the periodic shift on axis a."""
    dim = len(n)
    N = int(np.prod(n))
    idx = np.arange(N).reshape(shape_of(n))
    A = np.zeros((N, N))
    for a in range(dim):
        ax = dim - 1 - a  # numpy axis of grid axis a
        s = float(n[a]) ** 2
        for off in (+1, -1):
            nb = np.roll(idx, -off, axis=ax).reshape(-1)  # neighbour index of each point
            A[np.arange(N), nb] -= s
        A[np.arange(N), np.arange(N)] += 2 * s
    return A


def symbol_A(n):
    """Eigenvalues of periodic A on the Fourier grid, shaped like fftn output."""
    dim = len(n)
    lam = np.zeros(shape_of(n))
    for a in range(dim):
        ax = dim - 1 - a
        k = np.arange(n[a])
        la = float(n[a]) ** 2 * 4.0 * np.sin(np.pi * k / n[a]) ** 2
        sh = [1] * dim
        sh[ax] = n[a]
        lam = lam + la.reshape(sh)
    return lam


def spectral_A(n, v):
    lam = symbol_A(n)
    return np.real(np.fft.ifftn(lam * np.fft.fftn(v.reshape(shape_of(n))))).reshape(-1)


def dense_Ahat(n, y, eps, eyre=False):
    A = dense_A(n)
    D = np.diag(3 * y ** 2 - 1 + (1.0 if eyre else 0.0))
    return A @ (D + eps ** 2 * A)


def dense_ghat(n, y, eyre=False):
    A = dense_A(n)
    t = 2 * y ** 3 + (y if eyre else 0.0)
    return A @ t
