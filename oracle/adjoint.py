"""Gradient of the output-plane intensity with respect to per-cell
permittivity, FP64.  The paper has no gradient; this is the definition the
GPU adjoint is checked against.

Test infrastructure only (see the package docstring).

Loss: L(eps) = sum_f sum_plane |E_f(T)|^2, E_f the E components of the
response y_f(T) of eq. (ode) on the output plane.  Two routes:

* ``grad_fd``: central differences of L, each L from the exact response
  (augmented system, ``exact.y_plain``), with a Richardson step.
* ``grad_adjoint``: with lambda_f(t) = exp(-(T - t) A^T) lambda_f(T),
  lambda_f(T) = 2 P^T P y_f(T) (P picks the plane values),
      dL/deps_c = -sum_f int_0^T lambda_f(t)^T (dA/deps_c) y_f(t) dt,
  where A's E rows are (sigma E - curl H) / eps_node and eps_node is the mean
  of the cells around the node, so
      (dA/deps_c) y |_node = -(1 / (4 eps_node)) (A y)|_node
  for the E nodes whose closure holds cell c.  The time integral uses
  composite Gauss-Legendre quadrature on y(t), lambda(t) sampled by
  ``expm_multiply``.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import exact, yee


def loss(grid, eps_cell, g, omegas, T, plane):
    op = yee.Operator(grid, eps_cell)
    A = op.matrix()
    tot = 0.0
    for om in omegas:
        y = exact.y_plain(A, g, om, T)
        tot += yee.intensity(grid, y, plane)
    return tot


def grad_fd(grid, eps_cell, g, omegas, T, plane, cells, rel_step=1e-3):
    """Central differences at the given cells (flat indices), Richardson
    combination of steps h and h/2 (error O(h^4))."""
    eps_cell = np.asarray(eps_cell, np.float64)
    out = []
    for c in cells:
        e0 = eps_cell.reshape(-1)[c]
        vals = []
        for h in (rel_step * e0, 0.5 * rel_step * e0):
            ep = eps_cell.copy().reshape(-1)
            em = eps_cell.copy().reshape(-1)
            ep[c] += h
            em[c] -= h
            lp = loss(grid, ep.reshape(eps_cell.shape), g, omegas, T, plane)
            lm = loss(grid, em.reshape(eps_cell.shape), g, omegas, T, plane)
            vals.append((lp - lm) / (2 * h))
        out.append((4 * vals[1] - vals[0]) / 3)
    return np.array(out)


def plane_adjoint_seed(grid, y, plane):
    """lambda(T) = dL/dy = 2 P^T P y."""
    axis, idx = plane
    lam = np.zeros_like(y)
    nh = yee.n_h(grid.dim)
    for c in range(nh, grid.ncomp):
        F = y[c * grid.ncell:(c + 1) * grid.ncell].reshape(grid.shape)
        L = lam[c * grid.ncell:(c + 1) * grid.ncell].reshape(grid.shape)
        sl = [slice(None)] * grid.dim
        sl[grid.dim - 1 - axis] = idx
        L[tuple(sl)] = 2.0 * F[tuple(sl)]
    return lam


def cell_form(op, lam, y):
    """Per-cell lambda^T (dA/deps_c) y = -(1/4) sum over the E nodes e around
    cell c of lambda_e (A y)_e / eps_e."""
    grid = op.grid
    Ay = op.apply(y)
    nh = op.nh
    out = np.zeros(grid.shape)
    import itertools
    from .yee import offsets
    for c in range(nh, grid.ncomp):
        sl = slice(c * grid.ncell, (c + 1) * grid.ncell)
        q = (lam[sl] * Ay[sl]).reshape(grid.shape) / op.eps[c] * op.keep[c]
        off = offsets(grid.dim)[c]
        shifts = [[0] if off[a] == 0.5 else [0, 1] for a in range(grid.dim)]
        for combo in itertools.product(*shifts):
            t = q
            for a in range(grid.dim):
                if combo[a]:
                    # node (index) touches cell (index - 1): send to that cell
                    t = np.roll(t, -1, axis=grid.dim - 1 - a)
            out += t
    return -0.25 * out


def grad_adjoint(grid, eps_cell, g, omegas, T, plane, nsub=None, gauss=8):
    """dL/deps for every cell by the adjoint-state integral."""
    op = yee.Operator(grid, eps_cell)
    A = op.matrix()
    AT = A.T.tocsr()
    if nsub is None:
        nsub = max(8, int(np.ceil(T / 0.5)))
    xg, wg = np.polynomial.legendre.leggauss(gauss)
    grad = np.zeros(grid.shape)
    h = T / nsub
    ts = np.concatenate([(i + 0.5 * (xg + 1)) * h for i in range(nsub)])
    ws = np.concatenate([0.5 * h * wg for _ in range(nsub)])
    order = np.argsort(ts)
    ts, ws = ts[order], ws[order]
    for om in omegas:
        n = A.shape[0]
        eta = max(float(np.linalg.norm(g)), 1e-300)
        L = exact.augmented(A, g, om, eta)
        x0 = np.zeros(n + 2)
        x0[n + 1] = eta
        # y at every quadrature time, and y(T)
        ys = []
        x = x0
        tprev = 0.0
        for t in ts:
            x = spla.expm_multiply((t - tprev) * L, x)
            tprev = t
            ys.append(x[:n].copy())
        yT = spla.expm_multiply((T - tprev) * L, x)[:n]
        lamT = plane_adjoint_seed(grid, yT, plane)
        # lambda(t) = exp(-(T - t) A^T) lamT, marched backwards
        lam = lamT
        tnext = T
        lams = [None] * len(ts)
        for k in range(len(ts) - 1, -1, -1):
            lam = spla.expm_multiply(-(tnext - ts[k]) * AT, lam)
            tnext = ts[k]
            lams[k] = lam.copy()
        for k in range(len(ts)):
            grad -= ws[k] * cell_form(op, lams[k], ys[k])
    return grad
