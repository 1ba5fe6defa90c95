"""Exact solution of eq. (ode) with v = 0 and alpha(t) = sin(omega t), FP64.

Test infrastructure only (see the package docstring).

The method's target is y(T) = int_0^T exp(-(T - s) A) sin(omega s) g ds
(variation of constants, proof of eq. (split1)).  Two independent routes:

* ``y_plain``: the augmented homogeneous system of size n + 2 whose two
  extra states carry sin and cos of omega t, exponentiated by
  ``expm_multiply`` (Al-Mohy & Higham 2011).
* ``y_split``: eq. (split1), y(T) = Im(e^{i omega T} z) - exp(-T A) Im z with
  z = (A + i omega I)^{-1} g from a sparse LU solve.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def augmented(A, g, omega, eta=1.0):
    """Sparse L of size n + 2 with x' = L x, x = [y; eta sin; eta cos]:
    y' = -A y + (g / eta)(eta sin(omega t)), s' = omega c, c' = -omega s."""
    n = A.shape[0]
    col = sp.csr_matrix(np.asarray(g, np.float64).reshape(-1, 1) / eta)
    top = sp.hstack([-A, col, sp.csr_matrix((n, 1))])
    rot = sp.csr_matrix(np.array([[0.0, omega], [-omega, 0.0]]))
    bot = sp.hstack([sp.csr_matrix((2, n)), rot])
    return sp.vstack([top, bot]).tocsr()


def y_plain_pieces(A, g, omega, T, pieces, eta=None):
    """The augmented route of :func:`y_plain` one sub-interval at a time:
    yields (k, y(k T / pieces)) for k = 1 .. pieces, where y(t) is the first
    n entries of exp(t L) [0; 0; eta] and each step applies exp((T / pieces) L)
    to the previous state (the exponential is exact on every sub-interval)."""
    n = A.shape[0]
    if eta is None:
        eta = max(float(np.linalg.norm(g)), 1e-300)
    L = augmented(A, g, omega, eta)
    x = np.zeros(n + 2)
    x[n + 1] = eta
    dt = T / pieces
    for k in range(1, pieces + 1):
        x = spla.expm_multiply(dt * L, x)
        yield k, x[:n]


def y_plain(A, g, omega, T, eta=None, pieces=1):
    """y(T) from exp(T L) [0; 0; eta], L from :func:`augmented`.

    ``pieces`` splits [0, T] into equal sub-intervals (the exponential is
    exact on each one; this only bounds the work of one expm_multiply call).
    """
    y = None
    for _, y in y_plain_pieces(A, g, omega, T, pieces, eta):
        pass
    return y


def z_stat(A, g, omega):
    """z = (A + i omega I)^{-1} g (eq. (split1)), sparse LU."""
    n = A.shape[0]
    M = (A.astype(np.complex128) + 1j * omega * sp.identity(n, format="csr")).tocsc()
    return spla.spsolve(M, np.asarray(g, np.complex128))


def expm_action(A, T, b, pieces=1):
    """exp(-T A) b (eq. (y_homo))."""
    x = np.asarray(b, np.float64)
    dt = T / pieces
    for _ in range(pieces):
        x = spla.expm_multiply(-dt * A, x)
    return x


def y_split(A, g, omega, T, z=None, pieces=1):
    """y(T) = y~(T) - y^(T) with y~(T) = Im(e^{i omega T} z) and
    y^(T) = exp(-T A) Im z (eq. (split1), final sign '-')."""
    if z is None:
        z = z_stat(A, g, omega)
    ytil = np.imag(np.exp(1j * omega * T) * z)
    yhat = expm_action(A, T, np.imag(z), pieces)
    return ytil - yhat


def stationary_residual(apply_A, g, omega, z):
    """||g - (A + i omega I) z|| / ||g||, with A applied by the stencil."""
    r = np.asarray(g, np.complex128) - (apply_A(z.real) + 1j * apply_A(z.imag)) - 1j * omega * z
    return float(np.linalg.norm(r) / np.linalg.norm(g))
