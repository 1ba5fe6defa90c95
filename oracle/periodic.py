"""Two ways of using the time periodicity of the source (Sect. 3.5), plain
FP64.

Test infrastructure only (see the package docstring).

* ``split2`` -- source splitting, eq. (split2): restart in time on
  subintervals [(k-1) dT, k dT] with dT a whole number of source periods.
  On each subinterval y = w1 + w2 with w1' = -A w1, w1 = y((k-1) dT) at the
  start, and w2' = -A w2 + sin(W t) g, w2 = 0 at the start.  Because the
  source has the same phase at the start of every subinterval, w2 is the
  same on all of them and is solved once.  When T is not a multiple of dT,
  the last, shorter subinterval of length r uses w2 over [0, r] (again the
  same phase at its start).
* ``split1_next`` -- Fig. alg:spl1 with the neighbouring-frequency step
  (eq. (4diff)): for the first frequency the transient yhat(T) =
  exp(-T A) Im z is computed directly; for each next frequency
  yhat_next(T) = yhat(T) + w(T) with w' = -A w, w(0) = Im z_next - Im z.
"""
from __future__ import annotations

import math

import numpy as np

from . import exact


def split2(A, g, omega, T, dT):
    """y(T) by eq. (split2) with subinterval length dT (a multiple of
    2 pi / omega for the identity to hold)."""
    K = int(math.floor(T / dT + 1e-12))
    r = T - K * dT
    w2 = exact.y_plain(A, g, omega, dT)
    y = np.zeros(A.shape[0])
    for _ in range(K):
        y = exact.expm_action(A, dT, y) + w2
    if r > 1e-12 * T:
        y = exact.expm_action(A, r, y) + exact.y_plain(A, g, omega, r)
    return y


def period_multiple(omega, T, periods=1):
    """dT = periods * 2 pi / omega, at most T."""
    return min(T, periods * 2.0 * math.pi / omega)


def split1_next(A, g, omegas, T):
    """Responses y_j(T) for the frequencies in the given order by Fig.
    alg:spl1 steps 1-6.  Returns (responses, the norms ||w(0)|| of the
    difference problems, the norms ||Im z|| they replace)."""
    out, dnorms, znorms = [], [], []
    z_prev = None
    yhat_prev = None
    for W in omegas:
        z = exact.z_stat(A, g, W)
        ytil = np.imag(np.exp(1j * W * T) * z)
        if z_prev is None:
            yhat = exact.expm_action(A, T, np.imag(z))          # steps 1-3
        else:
            w0 = np.imag(z) - np.imag(z_prev)                    # step 4
            yhat = yhat_prev + exact.expm_action(A, T, w0)       # step 5, eq. (4diff)
            dnorms.append(float(np.linalg.norm(w0)))
            znorms.append(float(np.linalg.norm(np.imag(z))))
        out.append(ytil - yhat)                                  # final sign '-'
        z_prev, yhat_prev = z, yhat                              # step 6
    return out, dnorms, znorms
