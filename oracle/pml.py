"""The paper's 2D model with the perfectly matched layer (Sect. 2.1, eqs.
(mxw), (ode) with the auxiliary variable P), plain FP64.

Test infrastructure only (see the package docstring).

Fields y = [Hx, Hy, Ez, P] on the Yee grid of ``yee`` (2D), P on the Ez
nodes.  Eq. (mxw) with mu_r = 1, y' = -A y + alpha(t) g:

    Hx' = -dEz/dy
    Hy' =  dEz/dx - sigma Hy
    Ez' = (dHy/dx - dHx/dy) / eps - sigma Ez + P     (- J/eps)
    P'  = -(sigma / eps) dHx/dy

sigma = sigma_x(x) is nonzero only in the layers at both x ends and enters
Hy and Ez undivided by eps: this is the coordinate stretching
d/dx -> d/dx / (1 + i sigma / omega) written in time, where every field
decays at the same rate inside the layer and P carries the part of the
dHx/dy term the stretching does not touch.  sigma(d) = sigma_max (d/L)^2
with d the depth of the node's own x coordinate into the layer of L cells
(the quadratic profile of Sect. 4.1).  The discrete derivatives are those of
``yee``: dEz/dy, dEz/dx forward onto the H nodes, dHy/dx, dHx/dy backward
onto the Ez nodes.  In block form A = [[A_hat, B1^T], [-B2, 0]] (eq. (ode)):
B1^T = -I couples P into the Ez rows, -B2 = (sigma / eps) d/dy acts on Hx.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import yee


def _plain_grid(grid):
    """The same grid without P (for the masks, positions and eps of yee)."""
    return type(grid)(grid.dim, grid.n, grid.bc, grid.layer_axis, grid.layer_cells, grid.sigma_max)


def sigma_quadratic(grid, c):
    """sigma_max (d / L)^2 at the nodes of component c (0 Hx, 1 Hy, 2 Ez)."""
    g3 = _plain_grid(grid)
    L = float(grid.layer_cells)
    N = float(grid.n[0])
    x = yee.node_coords(g3, c)[0]
    d = np.maximum(np.maximum(L - x, x - (N - L)), 0.0)
    return grid.sigma_max * (d / L) ** 2


class PmlOperator:
    """The matrix A of eq. (ode) for the 2D model with the P variable."""

    def __init__(self, grid, eps_cell):
        assert grid.dim == 2 and grid.pml == 1 and grid.layer_axis == 0
        self.grid = grid
        g3 = _plain_grid(grid)
        self.g3 = g3
        self.eps_cell = np.asarray(eps_cell, np.float64)
        k3 = yee.keep_mask(g3)
        self.keep = k3 + [k3[2]]                       # P on the Ez nodes
        self.sig_hy = sigma_quadratic(grid, 1)
        self.sig_e = sigma_quadratic(grid, 2)
        self.eps = yee.eps_nodes(g3, self.eps_cell, 2)

    def apply(self, v):
        """w = A v from the component equations above."""
        g3 = self.g3
        nc = g3.ncell
        comps = [np.asarray(v, np.float64)[c * nc:(c + 1) * nc].reshape(g3.shape) * self.keep[c]
                 for c in range(4)]
        Hx, Hy, Ez, P = comps
        fwd, bwd = yee._fwd, yee._bwd
        out = [
            fwd(Ez, 2, 1) - Ez,                                           # -Hx'
            self.sig_hy * Hy - (fwd(Ez, 2, 0) - Ez),                      # -Hy'
            -((Hy - bwd(Hy, 2, 0)) - (Hx - bwd(Hx, 2, 1))) / self.eps + self.sig_e * Ez - P,
            self.sig_e / self.eps * (Hx - bwd(Hx, 2, 1)),                 # -P'
        ]
        return np.concatenate([(o * k).reshape(-1) for o, k in zip(out, self.keep)])

    def matrix(self):
        """A assembled as [[A_hat, B1^T], [-B2, 0]] from yee's curl matrix."""
        g3 = self.g3
        nc = g3.ncell
        K = yee.Operator(g3, self.eps_cell).curl_matrix()      # rows (Hx, Hy), column Ez
        inv_eps = sp.diags(1.0 / self.eps.reshape(-1))
        Z = sp.csr_matrix((nc, nc))
        SH = sp.diags(np.concatenate([np.zeros(nc), self.sig_hy.reshape(-1)]))
        SE = sp.diags(self.sig_e.reshape(-1))
        A_hat = sp.bmat([[SH, K], [-inv_eps @ K.T, SE]], format="csr")
        # d/dy backward onto the Ez nodes, acting on Hx
        I = sp.identity(nc, format="csr")
        Dy_b = I - yee.Operator(g3, self.eps_cell)._shift(1).T
        B1T = sp.bmat([[Z], [Z], [-I]], format="csr")
        mB2 = sp.bmat([[sp.diags(self.sig_e.reshape(-1)) @ inv_eps @ Dy_b, Z, Z]], format="csr")
        A = sp.bmat([[A_hat, B1T], [mB2, Z]], format="csr")
        keep = sp.diags(np.concatenate([k.reshape(-1) for k in self.keep]))
        return (keep @ A @ keep).tocsr()

    def apply_T(self, w):
        """A^T w by the library transpose of the assembled matrix."""
        return self.matrix().T @ np.asarray(w, np.float64)
