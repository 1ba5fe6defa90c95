"""Pins of the PML oracle (eq. (mxw) with the auxiliary variable P, the
block form A = [[A_hat, B1^T], [-B2, 0]] of eq. (ode), the quadratic
profile of Sect. 4.1) against facts fixed outside it."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import scenario as S
from oracle import pml, yee


def _grid(bc=(S.PEC, S.PEC), n=(23, 17), L=4, smax=2.0):
    return S.Grid(2, n, bc, 0, L, smax, pml=1)


def _eps(grid, seed=4):
    return 1.0 + 2.0 * np.random.default_rng(seed).random(grid.shape)


@pytest.mark.parametrize("bc", [(S.PEC, S.PEC), (S.PEC, S.PERIODIC), (S.PERIODIC, S.PERIODIC)])
def test_component_formulas_equal_block_matrix(bc):
    grid = _grid(bc)
    op = pml.PmlOperator(grid, _eps(grid))
    v = S.masked_random_vector(grid, 3)
    assert np.allclose(op.apply(v), op.matrix() @ v, rtol=0, atol=1e-13 * np.abs(v).max() * 10)


def test_without_conductivity_the_maxwell_block_is_the_plain_operator():
    """sigma_max = 0: the [H; E] block is the lossless Yee operator of
    eq. (ode), P feeds Ez with -1 and is fed by nothing."""
    grid = _grid(smax=0.0)
    eps = _eps(grid)
    A = pml.PmlOperator(grid, eps).matrix().toarray()
    g3 = S.Grid(2, grid.n, grid.bc, 0, grid.layer_cells, 0.0)
    B = yee.Operator(g3, eps).matrix().toarray()
    nc = grid.ncell
    assert np.abs(A[:3 * nc, :3 * nc] - B).max() < 1e-15
    assert not np.any(A[3 * nc:, :])
    keepE = S.wall_keep_mask(g3).reshape(3, nc)[2]
    assert np.array_equal(A[2 * nc:3 * nc, 3 * nc:], -np.diag(keepE))


def test_quadratic_profile_values():
    """sigma_max (d/L)^2 at the Hy nodes (x = i + 1/2) and Ez nodes (x = i),
    written out for every i; Hx is not damped."""
    grid = _grid(n=(23, 5), L=4, smax=2.0)
    nx, L = 23, 4.0
    want_hy = [2.0 * (max(L - (i + 0.5), (i + 0.5) - (nx - L), 0.0) / L) ** 2 for i in range(nx)]
    want_e = [2.0 * (max(L - i, i - (nx - L), 0.0) / L) ** 2 for i in range(nx)]
    assert np.allclose(pml.sigma_quadratic(grid, 1)[0], want_hy, atol=1e-15)
    assert np.allclose(pml.sigma_quadratic(grid, 2)[0], want_e, atol=1e-15)
    A = pml.PmlOperator(grid, _eps(grid)).matrix()
    nc = grid.ncell
    assert np.abs(A[:nc, :nc]).max() == 0.0           # no Hx damping


def test_eliminating_P_gives_the_stretched_coordinate_system():
    """The defining property of the layer: at a frequency W, eliminating P
    from (A + iW) z = g leaves Maxwell's equations with every x-difference
    divided by the local stretching s = 1 + sigma / (iW) (the y-differences
    untouched) and the source divided by s on the Ez nodes.  The stretched
    system is written here from that definition with its own difference
    matrices."""
    nx, ny = 26, 14
    grid = _grid(bc=(S.PERIODIC, S.PERIODIC), n=(nx, ny), L=5, smax=1.7)
    eps_cell = _eps(grid, 9)
    op = pml.PmlOperator(grid, eps_cell)
    W = 0.83
    nc = grid.ncell
    rng = np.random.default_rng(2)
    gE = rng.standard_normal(nc)
    g = np.zeros(4 * nc)
    g[2 * nc:3 * nc] = gE
    z = spla.spsolve((op.matrix().astype(complex) + 1j * W * sp.identity(4 * nc)).tocsc(), g.astype(complex))

    def shift(dx, dy):        # (S f)[j, i] = f[j + dy, i + dx], periodic
        idx = np.arange(nc).reshape(ny, nx)
        src = np.roll(np.roll(idx, -dy, axis=0), -dx, axis=1).reshape(-1)
        return sp.csr_matrix((np.ones(nc), (np.arange(nc), src)), shape=(nc, nc))

    I = sp.identity(nc)
    Dxf, Dyf = shift(1, 0) - I, shift(0, 1) - I
    Dxb, Dyb = I - shift(-1, 0), I - shift(0, -1)
    e = eps_cell
    eps_node = (e + np.roll(e, 1, 1) + np.roll(e, 1, 0) + np.roll(np.roll(e, 1, 0), 1, 1)).reshape(-1) / 4
    x = np.arange(nx, dtype=float)
    depth = lambda p: np.maximum(np.maximum(5.0 - p, p - (nx - 5.0)), 0.0)
    sig_h = np.tile(1.7 * (depth(x + 0.5) / 5.0) ** 2, ny)
    sig_e = np.tile(1.7 * (depth(x) / 5.0) ** 2, ny)
    sH = 1.0 + sig_h / (1j * W)
    sE = 1.0 + sig_e / (1j * W)
    D = sp.diags
    M = sp.bmat([[1j * W * I, None, Dyf],
                 [None, 1j * W * I, -D(1.0 / sH) @ Dxf],
                 [D(1.0 / eps_node) @ Dyb, -D(1.0 / (eps_node * sE)) @ Dxb, 1j * W * I]], format="csc")
    rhs = np.concatenate([np.zeros(2 * nc), gE / sE])
    u = spla.spsolve(M, rhs)
    assert np.linalg.norm(z[:3 * nc] - u) <= 1e-10 * np.linalg.norm(u)


def test_normally_incident_pulse_is_absorbed():
    """A y-independent pulse in eps = 2.25 runs into the layers at both x
    ends: after it has entered them, the interior keeps < 1e-6 of the
    energy.  The same profile with sigma / eps in the Ez rows (a layer whose
    E and H decay at different rates) reflects > 1e-2."""
    nx, ny, L = 100, 8, 10
    grid = S.Grid(2, (nx, ny), (S.PEC, S.PERIODIC), 0, L, 1.5, pml=1)
    op = pml.PmlOperator(grid, np.full(grid.shape, 2.25))
    nc = grid.ncell
    A = op.matrix()
    fix = sp.diags(np.concatenate([np.zeros(2 * nc), -op.sig_e.reshape(-1) + op.sig_e.reshape(-1) / 2.25,
                                   np.zeros(nc)]))
    x = np.arange(nx)[None, :] * np.ones((ny, 1))
    v = np.zeros(4 * nc)
    v[2 * nc:3 * nc] = np.exp(-((x - nx / 2) / 4.0) ** 2).reshape(-1)

    def interior_energy(u):
        Hx, Hy, E = (u[c * nc:(c + 1) * nc].reshape(ny, nx)[:, L + 2:nx - L - 2] for c in range(3))
        return float((Hx ** 2 + Hy ** 2 + 2.25 * E ** 2).sum())

    e0 = interior_energy(v)
    good = interior_energy(spla.expm_multiply(-90.0 * A, v)) / e0
    bad = interior_energy(spla.expm_multiply(-90.0 * (A + fix), v)) / e0
    assert good < 1e-6
    assert bad > 1e-2
