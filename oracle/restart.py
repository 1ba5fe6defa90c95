"""Residual-based restarting in Krylov dimension for many source
frequencies at once (Sect. 3.4, eq. (rst), Corollary 2, Fig. alg:rst),
regular (not shift-and-invert) Krylov variant, plain FP64.

Test infrastructure only (see the package docstring).

The method.  After m Arnoldi steps from v_1 = g / ||g||, the projected
problem (eq. (corr2)) u' = -H_m u + alpha(t) beta e_1, u(0) = 0, gives the
iterate y_m(t) = V_m u(t), whose residual is r_m(t) = alphahat(t) v_{m+1}
with alphahat(t) = -h_{m+1,m} e_m^T u(t) (eq. (resid)).  Restarting
(eq. (rst)) keeps y_m as the new initial guess and solves for the
correction with source alphahat(t) v_{m+1}: a new Arnoldi process from
v_{m+1} (norm 1, so beta = 1 from then on) and a new projected problem
driven by alphahat.  The Krylov basis never depends on alpha (Corollary 2),
so one basis per restart serves every frequency; only the projected
problems are per frequency (Fig. alg:rst, steps (1)-(3)).

How this oracle holds alphahat.  Fig. alg:rst samples and stores alphahat
per frequency; here each alphahat is kept exactly instead, as the output of
a linear system: x' = L x, x(0) = x0, alphahat(t) = c^T x(t).  For the
first restart x = (sin W t, cos W t) and c = (beta, 0).  Each restart
appends the new projected state u to x,

    L <- [[L, 0], [e_1 c^T, -H_m]],   x0 <- [x0; 0],   c <- [0; -h_{m+1,m} e_m],

so u(t) of every restart is an exact matrix exponential of the stacked
system (no time discretisation), and the stopping test (step 2(c)) reads
max_t |alphahat(t)| on a uniform grid of ``nsample`` points.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .krylov import arnoldi


def _sample_max(L, x0, c, T, nsample):
    """max over t_i = i T / nsample (i = 0..nsample) of |c^T exp(t_i L) x0|."""
    E = sla.expm((T / nsample) * L)
    x = x0.copy()
    mx = abs(float(c @ x))
    for _ in range(nsample):
        x = E @ x
        mx = max(mx, abs(float(c @ x)))
    return mx


def restart_dim(apply_A, g, omegas, T, m, max_restarts=200, rtol=1e-10, nsample=400, t_eval=()):
    """y(T) of eq. (ode), y' = -A y + sin(W t) g, y(0) = 0, for every W in
    ``omegas`` by Fig. alg:rst (regular Krylov variant).

    A frequency stops (step 2(c)) after the first restart whose new residual
    satisfies max_t |alphahat(t)| ||v_{m+1}|| <= rtol * ||g||.  The loop ends
    when every frequency has stopped or after ``max_restarts`` restarts.

    Returns a dict with
      y         list of y(T) per frequency,
      y_t       per frequency, the iterate y(t) at each time in ``t_eval``,
      restarts  per frequency, restarts made,
      resid     per frequency, the last max_t |alphahat(t)|,
      alpha     per frequency, (L, x0, c) of the last alphahat,
      v_next    the last v_{m+1} (the residual direction),
      converged per frequency.
    """
    g = np.asarray(g, np.float64)
    omegas = list(omegas)
    nf = len(omegas)
    beta = float(np.linalg.norm(g))
    n = g.size
    out = {"y": [np.zeros(n) for _ in omegas], "y_t": [[np.zeros(n) for _ in t_eval] for _ in omegas],
           "restarts": [0] * nf, "resid": [0.0] * nf, "alpha": [None] * nf, "v_next": None,
           "converged": [beta == 0.0] * nf}
    if beta == 0.0:
        return out
    # source realisations alpha_1(t) = beta sin(W t)
    real = []
    for W in omegas:
        L = np.array([[0.0, W], [-W, 0.0]])
        real.append((L, np.array([0.0, 1.0]), np.array([beta, 0.0])))
    active = [True] * nf
    v = g / beta
    for k in range(max_restarts):
        if not any(active):
            break
        # step (1): m Arnoldi steps, shared by every frequency
        V, H, _, md = arnoldi(apply_A, v, m)
        Hm = H[:md, :md]
        hnext = float(H[md, md - 1])
        for f in range(nf):
            if not active[f]:
                continue
            L, x0, c = real[f]
            q = L.shape[0]
            # step 2(a): u' = -H_m u + alphahat(t) e_1, u(0) = 0, stacked
            Ln = np.zeros((q + md, q + md))
            Ln[:q, :q] = L
            Ln[q, :q] = c
            Ln[q:, q:] = -Hm
            xn = np.concatenate([x0, np.zeros(md)])
            uT = (sla.expm(T * Ln) @ xn)[q:]
            # step (3) for this frequency: y(T) += V_m u(T)
            out["y"][f] += V[:, :md] @ uT
            for i, t in enumerate(t_eval):
                out["y_t"][f][i] += V[:, :md] @ (sla.expm(t * Ln) @ xn)[q:]
            # step 2(b): alphahat(t) = -h_{m+1,m} e_m^T u(t)
            cn = np.zeros(q + md)
            cn[q + md - 1] = -hnext
            real[f] = (Ln, xn, cn)
            out["alpha"][f] = real[f]
            out["restarts"][f] = k + 1
            # step 2(c)
            r = 0.0 if hnext == 0.0 else _sample_max(Ln, xn, cn, T, nsample)
            out["resid"][f] = r
            if r <= rtol * beta:
                active[f] = False
                out["converged"][f] = True
        # step (3): the next basis starts from v_{m+1}
        v = V[:, md]
        out["v_next"] = v.copy()
        if hnext == 0.0:
            # invariant subspace: every projection is exact
            for f in range(nf):
                active[f] = False
                out["converged"][f] = True
            break
    return out


def alpha_at(real, t):
    """alphahat(t) = c^T exp(t L) x0 of a realisation (L, x0, c)."""
    L, x0, c = real
    return float(c @ (sla.expm(t * L) @ x0))
