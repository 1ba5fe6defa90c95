"""Krylov-subspace pieces of the method, plain FP64.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def arnoldi(apply_A, v0, m, breakdown_tol=1e-12):
    """m steps of the Arnoldi process for K_m(A, v0) (Sect. 3.2, eqs. (Arn),
    (Krylov)), modified Gram-Schmidt in the Euclidean inner product.

    Returns (V, H, beta, m_done): V is n x (m_done + 1) with orthonormal
    columns, v_1 = v0 / ||v0||; H is the (m_done + 1) x m_done upper
    Hessenberg matrix with A V_m = V_{m+1} H; beta = ||v0||.  A lucky
    breakdown (h_{j+1,j} <= breakdown_tol * max_i ||A v_i||) stops early;
    then the last column of V is zero and H's last row is zero.
    """
    v0 = np.asarray(v0, np.float64)
    n = v0.size
    beta = float(np.linalg.norm(v0))
    V = np.zeros((n, m + 1))
    H = np.zeros((m + 1, m))
    V[:, 0] = v0 / beta
    scale = 0.0
    for j in range(m):
        w = apply_A(V[:, j])
        scale = max(scale, float(np.linalg.norm(w)))
        for i in range(j + 1):
            H[i, j] = V[:, i] @ w
            w = w - H[i, j] * V[:, i]
        h = float(np.linalg.norm(w))
        H[j + 1, j] = h
        if h <= breakdown_tol * scale:
            H[j + 1, j] = 0.0
            return V[:, :j + 2] * np.r_[np.ones(j + 1), 0.0], H[:j + 2, :j + 1], beta, j + 1
        V[:, j + 1] = w / h
    return V, H, beta, m


def proj_exp(H, tau, beta):
    """u(tau) = exp(-tau H_m) beta e_1: the homogeneous projected problem
    u' = -H_m u, u(0) = beta e_1 (eq. (corr2) with alpha = 0 and a nonzero
    initial value, Sect. 4.1 'expm' for the homogeneous case)."""
    m = H.shape[1]
    e1 = np.zeros(m)
    e1[0] = beta
    return sla.expm(-tau * H[:m, :m]) @ e1


def proj_sine(H, beta, omega, T):
    """u(T) of eq. (corr2) with alpha(t) = sin(omega t):
    u' = -H_m u + sin(omega t) beta e_1, u(0) = 0.

    Solved exactly as a homogeneous system of size m + 2: the two extra
    states (s, c) obey s' = omega c, c' = -omega s, s(0) = 0, c(0) = 1, so
    s(t) = sin(omega t), and u' = -H u + s beta e_1."""
    m = H.shape[1]
    N = np.zeros((m + 2, m + 2))
    N[:m, :m] = -H[:m, :m]
    N[0, m] = beta
    N[m, m + 1] = omega
    N[m + 1, m] = -omega
    x0 = np.zeros(m + 2)
    x0[m + 1] = 1.0
    return (sla.expm(T * N) @ x0)[:m]


def phi1_times(X, b):
    """phi_1(X) b = X^{-1}(e^X - I) b from the exponential of the augmented
    matrix [[X, b], [0, 0]] (Saad 1992, 'Analysis of some Krylov subspace
    approximations to the matrix exponential operator', Sect. 2)."""
    m = X.shape[0]
    Z = np.zeros((m + 1, m + 1), dtype=np.result_type(X, b))
    Z[:m, :m] = X
    Z[:m, m] = b
    return sla.expm(Z)[:m, m]


def proj_sine_phi(H, beta, omega, T):
    """The same u(T) as :func:`proj_sine`, by the phi route:
    u(T) = Im[ e^{i omega T} T phi_1(-T (H + i omega I)) beta e_1 ]
    (variation of constants, as in the proof of eq. (split1))."""
    m = H.shape[1]
    Hm = H[:m, :m].astype(np.complex128)
    X = -T * (Hm + 1j * omega * np.eye(m))
    b = np.zeros(m, np.complex128)
    b[0] = beta
    return np.imag(np.exp(1j * omega * T) * T * phi1_times(X, b))


def shifted_solve(H, omega, rho):
    """c = rho (H_m + i omega I)^{-1} e_1: the projected stationary system of
    the shifted full orthogonalisation method for (A + i omega I) z = r,
    r = rho v_1 (shift invariance of K_m(A, v_1))."""
    m = H.shape[1]
    rhs = np.zeros(m, np.complex128)
    rhs[0] = rho
    return np.linalg.solve(H[:m, :m] + 1j * omega * np.eye(m), rhs)


def lemma1_residual(H, u, v_next):
    """r_m = -h_{m+1,m} (e_m^T u) v_{m+1} (Lemma 1, eq. (resid), regular
    Krylov)."""
    m = H.shape[1]
    return -H[m, m - 1] * u[m - 1] * v_next


def shifted_fom(apply_A, g, omegas, m, rtol, max_cycles=500):
    """Restarted shifted FOM for (A + i omega_j I) z_j = g, all j on one basis.

    Each cycle runs m Arnoldi steps from the common residual direction; the
    residual of every shift is collinear with v_{m+1} (eq. (Arn1)), so the
    next cycle restarts from v_{m+1} with per-shift coefficients rho_j
    (Simoncini 2003, 'Restarted full orthogonalization method for shifted
    linear systems').  Returns (z, rel_resid, cycles)."""
    g = np.asarray(g, np.float64)
    n = g.size
    nf = len(omegas)
    beta = float(np.linalg.norm(g))
    z = np.zeros((nf, n), np.complex128)
    rho = np.full(nf, beta, np.complex128)
    v = g / beta
    for cyc in range(max_cycles):
        V, H, _, md = arnoldi(apply_A, v, m)
        for j, om in enumerate(omegas):
            c = shifted_solve(H, om, rho[j])
            z[j] += V[:, :md] @ c
            rho[j] = -H[md, md - 1] * c[md - 1]
        if np.max(np.abs(rho)) <= rtol * beta or H[md, md - 1] == 0.0:
            return z, np.abs(rho) / beta, cyc + 1
        v = V[:, md]
    return z, np.abs(rho) / beta, max_cycles
