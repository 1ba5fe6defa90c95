"""Semi-discrete Yee-grid Maxwell operator A of eq. (ode), in plain FP64 numpy.

Test infrastructure only (see the package docstring).

Model (Sect. 2.1, eqs. (mxw), (ode)): dimensionless Maxwell equations with
mu_r = 1, a piecewise-constant eps_r and an absorbing conductivity sigma.
After Yee discretisation in space the fields y = [H; E] obey
``y' = -A y + alpha(t) g`` with

    A = diag(M_mu, M_eps)^{-1} [[ M_sigma,  K      ],
                                [ -K^T,     M_sigma ]]

(the matrix A-hat of eq. (ode); the PML auxiliary variable P is not
modelled, the absorbing layer is a plain lossy layer).  K is the discrete
curl of E evaluated on the H nodes, K^T the discrete curl of H on the E
nodes.  Written per component, the rows of A are

    H rows:  (A y)_H = sigma_H * H + (curl E)_H          (mu = 1)
    E rows:  (A y)_E = (sigma_E * E - (curl H)_E) / eps_E

so that H' = -curl E - sigma H and eps E' = curl H - sigma E - J, the
component equations of eq. (mxw).

Readings of the paper used here (all listed in the design notes):
* sigma enters the E rows divided by eps (the matrix form of eq. (ode); eq.
  (mxw) writes sigma_x E_z without the 1/eps) and damps every component
  inside the layer, not only H_y and E_z.
* 2D field set (H_x, H_y, E_z), E on grid vertices and H on edge centres, as
  the paper states below eq. (ic1); 3D uses the textbook Yee cell.
* eps on an E node is the arithmetic mean of the permittivities of the
  cells whose closure contains the node (4 cells in 3D and in 2D).
* A perfectly conducting wall at index 0 of an axis (index n wraps onto it)
  removes every node with an integer coordinate along that axis there: the
  tangential E and the normal H.  Those entries of A (rows and columns) are
  zero.
* sigma(d) = sigma_max * d / L, with d the depth of the node's own
  (staggered) coordinate into the layer of thickness L at either end.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

PEC = 1


def offsets(dim):
    """Per-component staggered offsets along (x, y[, z]).

    2D order (Hx, Hy, Ez): Ez at vertices (0, 0); Hx at the centre of the
    y-directed edge (0, 1/2); Hy at the centre of the x-directed edge
    (1/2, 0).  3D order (Hx, Hy, Hz, Ex, Ey, Ez): H_c at face centres,
    E_c at edge centres of the Yee cell.
    """
    if dim == 2:
        return [(0.0, 0.5), (0.5, 0.0), (0.0, 0.0)]
    return [(0.0, 0.5, 0.5), (0.5, 0.0, 0.5), (0.5, 0.5, 0.0),
            (0.5, 0.0, 0.0), (0.0, 0.5, 0.0), (0.0, 0.0, 0.5)]


def n_h(dim):
    return 2 if dim == 2 else 3


def node_coords(grid, c):
    """Coordinates of every node of component c, as arrays of grid.shape."""
    dim = grid.dim
    axes = [np.arange(grid.n[a]) + offsets(dim)[c][a] for a in range(dim)]
    mesh = np.meshgrid(*reversed(axes), indexing="ij")   # slowest first
    return list(reversed(mesh))                            # (x, y[, z])


def keep_mask(grid):
    """Per-component 0/1 arrays: 0 where the node lies on a conducting wall."""
    dim = grid.dim
    out = []
    for c in range(grid.ncomp):
        k = np.ones(grid.shape)
        for a in range(dim):
            if grid.bc[a] == PEC and offsets(dim)[c][a] == 0.0:
                sl = [slice(None)] * dim
                sl[dim - 1 - a] = 0
                k[tuple(sl)] = 0.0
        out.append(k)
    return out


def sigma_nodes(grid, c):
    """Conductivity at the nodes of component c: linear ramp in the layer."""
    a = grid.layer_axis
    L = float(grid.layer_cells)
    N = float(grid.n[a])
    pos = node_coords(grid, c)[a]
    d = np.maximum(np.maximum(L - pos, pos - (N - L)), 0.0)
    return grid.sigma_max * d / L


def eps_nodes(grid, eps_cell, c):
    """Permittivity on the nodes of E component c: mean of the touching cells.

    Along an axis where the node coordinate is half-integer the node lies
    inside cell ``index``; where it is integer the node lies on the face
    shared by cells ``index - 1`` and ``index`` (periodic wrap).
    """
    dim = grid.dim
    off = offsets(dim)[c]
    acc = np.zeros(grid.shape)
    cnt = 0
    shifts = [[0] if off[a] == 0.5 else [0, 1] for a in range(dim)]
    import itertools
    for combo in itertools.product(*shifts):
        e = eps_cell
        for a in range(dim):
            if combo[a]:
                e = np.roll(e, 1, axis=dim - 1 - a)   # value of cell index-1
        acc = acc + e
        cnt += 1
    return acc / cnt


def _fwd(F, dim, a):
    """F at index + e_a (periodic)."""
    return np.roll(F, -1, axis=dim - 1 - a)


def _bwd(F, dim, a):
    """F at index - e_a (periodic)."""
    return np.roll(F, 1, axis=dim - 1 - a)


def split(grid, v):
    return [v[c * grid.ncell:(c + 1) * grid.ncell].reshape(grid.shape)
            for c in range(grid.ncomp)]


def curl_E(grid, E):
    """Discrete curl of E on the H nodes (the K of eq. (ode))."""
    dim = grid.dim
    if dim == 2:
        (Ez,) = E
        # curl (Ez z^) = (dEz/dy, -dEz/dx)
        return [_fwd(Ez, 2, 1) - Ez, -(_fwd(Ez, 2, 0) - Ez)]
    Ex, Ey, Ez = E
    cx = (_fwd(Ez, 3, 1) - Ez) - (_fwd(Ey, 3, 2) - Ey)
    cy = (_fwd(Ex, 3, 2) - Ex) - (_fwd(Ez, 3, 0) - Ez)
    cz = (_fwd(Ey, 3, 0) - Ey) - (_fwd(Ex, 3, 1) - Ex)
    return [cx, cy, cz]


def curl_H(grid, H):
    """Discrete curl of H on the E nodes (the K^T of eq. (ode))."""
    dim = grid.dim
    if dim == 2:
        Hx, Hy = H
        return [(Hy - _bwd(Hy, 2, 0)) - (Hx - _bwd(Hx, 2, 1))]
    Hx, Hy, Hz = H
    cx = (Hz - _bwd(Hz, 3, 1)) - (Hy - _bwd(Hy, 3, 2))
    cy = (Hx - _bwd(Hx, 3, 2)) - (Hz - _bwd(Hz, 3, 0))
    cz = (Hy - _bwd(Hy, 3, 0)) - (Hx - _bwd(Hx, 3, 1))
    return [cx, cy, cz]


class Operator:
    """The matrix A of eq. (ode) for one grid and one permittivity field."""

    def __init__(self, grid, eps_cell):
        self.grid = grid
        self.eps_cell = np.asarray(eps_cell, dtype=np.float64)
        nh = n_h(grid.dim)
        self.nh = nh
        self.keep = keep_mask(grid)
        self.sigma = [sigma_nodes(grid, c) for c in range(grid.ncomp)]
        self.eps = [None] * nh + [eps_nodes(grid, self.eps_cell, c)
                                  for c in range(nh, grid.ncomp)]

    @property
    def n(self):
        return self.grid.nunk

    def keep_vector(self):
        return np.concatenate([k.reshape(-1) for k in self.keep])

    def apply(self, v):
        """w = A v, component formulas of eq. (mxw)."""
        g = self.grid
        comps = [f * k for f, k in zip(split(g, np.asarray(v, np.float64)), self.keep)]
        H, E = comps[:self.nh], comps[self.nh:]
        cE = curl_E(g, E)
        cH = curl_H(g, H)
        out = []
        for c in range(self.nh):
            out.append((self.sigma[c] * H[c] + cE[c]) * self.keep[c])
        for q in range(len(E)):
            c = self.nh + q
            out.append((self.sigma[c] * E[q] - cH[q]) / self.eps[c] * self.keep[c])
        return np.concatenate([o.reshape(-1) for o in out])

    def apply_T(self, w):
        """A^T w, from the matrix form: A^T = [[S, -K],[K^T, S]] M^{-1}."""
        g = self.grid
        comps = [f * k for f, k in zip(split(g, np.asarray(w, np.float64)), self.keep)]
        Hs = comps[:self.nh]
        Es = [comps[self.nh + q] / self.eps[self.nh + q] for q in range(len(comps) - self.nh)]
        cE = curl_E(g, Es)       # K (M_eps^{-1} w_E)
        cH = curl_H(g, Hs)       # K^T w_H
        out = []
        for c in range(self.nh):
            out.append((self.sigma[c] * Hs[c] - cE[c]) * self.keep[c])
        for q in range(len(Es)):
            c = self.nh + q
            out.append((self.sigma[c] * Es[q] + cH[q]) * self.keep[c])
        return np.concatenate([o.reshape(-1) for o in out])

    # --- assembled form: the block matrix of eq. (ode) --------------------
    def _shift(self, a):
        """Sparse S with (S F)[idx] = F[idx + e_a] (periodic), one component."""
        g = self.grid
        dim = g.dim
        mats = []
        for b in reversed(range(dim)):    # slowest axis first (kron order)
            nb = g.n[b]
            if b == a:
                mats.append(sp.diags([np.ones(nb - 1), np.ones(1)], [1, -(nb - 1)],
                                     shape=(nb, nb), format="csr"))
            else:
                mats.append(sp.identity(nb, format="csr"))
        S = mats[0]
        for M in mats[1:]:
            S = sp.kron(S, M, format="csr")
        return S

    def curl_matrix(self):
        """K: E -> H nodes, assembled from forward differences D_a = S_a - I."""
        g = self.grid
        nc = g.ncell
        I = sp.identity(nc, format="csr")
        D = [self._shift(a) - I for a in range(g.dim)]
        Z = sp.csr_matrix((nc, nc))
        if g.dim == 2:
            # rows (Hx, Hy), column Ez
            return sp.bmat([[D[1]], [-D[0]]], format="csr")
        return sp.bmat([[Z, -D[2], D[1]],
                        [D[2], Z, -D[0]],
                        [-D[1], D[0], Z]], format="csr")

    def matrix(self):
        """A = M^{-1} [[Sigma_H, K], [-K^T, Sigma_E]] restricted to the kept nodes."""
        K = self.curl_matrix()
        SH = sp.diags(np.concatenate([s.reshape(-1) for s in self.sigma[:self.nh]]))
        SE = sp.diags(np.concatenate([s.reshape(-1) for s in self.sigma[self.nh:]]))
        core = sp.bmat([[SH, K], [-K.T, SE]], format="csr")
        Minv = sp.diags(1.0 / self.weights())
        P = sp.diags(self.keep_vector())
        return (P @ Minv @ core @ P).tocsr()

    def weights(self):
        """Diagonal of M = diag(M_mu, M_eps): 1 on H nodes, eps on E nodes."""
        parts = [np.ones(self.grid.ncell)] * self.nh
        parts += [self.eps[c].reshape(-1) for c in range(self.nh, self.grid.ncomp)]
        return np.concatenate(parts)

    def sigma_vector(self):
        return np.concatenate([s.reshape(-1) for s in self.sigma])


def plane_fields(grid, y, plane):
    """E components on the output plane, shape (n_E, plane nodes).

    ``plane = (axis, index)``.  2D: E_z on the line x = index.  3D: E_x, E_y
    at z = index and E_z at z = index + 1/2.
    """
    axis, idx = plane
    comps = split(grid, y)
    nh = n_h(grid.dim)
    out = []
    for c in range(nh, grid.ncomp):
        F = comps[c]
        sl = [slice(None)] * grid.dim
        sl[grid.dim - 1 - axis] = idx
        out.append(F[tuple(sl)].reshape(-1))
    return np.stack(out)


def intensity(grid, y, plane):
    """Summed |E|^2 over the output plane."""
    P = plane_fields(grid, y, plane)
    return float((P * P).sum())
