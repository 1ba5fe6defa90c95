"""Pins of the oracle gradient (dL/d eps per cell of the summed output-plane
intensity): the adjoint-state integral against central differences of the
exact forward solve, and the per-cell operator derivative against central
differences of the operator itself."""
import numpy as np
import pytest

import scenario as S
from oracle import adjoint, yee


@pytest.mark.parametrize("cfg", ["2d", "3d"])
def test_adjoint_integral_matches_finite_differences(cfg):
    sc = S.config_2d(n=10, ndisks=2, T=6.0) if cfg == "2d" else S.config_3d(n=6, fill=0.3, T=4.0)
    eps = sc.eps_cell * (1.0 + 0.3 * np.random.default_rng(3).random(sc.grid.shape))
    oms = S.freq_list(2)
    ga = adjoint.grad_adjoint(sc.grid, eps, sc.g, oms, sc.T, sc.plane)
    cells = np.random.default_rng(5).choice(eps.size, 6, replace=False)
    gf = adjoint.grad_fd(sc.grid, eps, sc.g, oms, sc.T, sc.plane, cells)
    assert np.abs(ga.reshape(-1)[cells] - gf).max() < 1e-8 * np.abs(gf).max()


def test_cell_form_is_the_operator_derivative():
    """lambda^T (dA/deps_c) y from the closed form equals the central
    difference of lambda^T A(eps) y in eps_c."""
    sc = S.config_3d(n=6, fill=0.3)
    eps = 1.0 + np.random.default_rng(1).random(sc.grid.shape)
    lam = S.masked_random_vector(sc.grid, 2)
    y = S.masked_random_vector(sc.grid, 3)
    form = adjoint.cell_form(yee.Operator(sc.grid, eps), lam, y)
    for c in np.random.default_rng(4).choice(eps.size, 8, replace=False):
        h = 1e-5
        ep = eps.copy().reshape(-1); ep[c] += h
        em = eps.copy().reshape(-1); em[c] -= h
        fp = lam @ yee.Operator(sc.grid, ep.reshape(eps.shape)).apply(y)
        fm = lam @ yee.Operator(sc.grid, em.reshape(eps.shape)).apply(y)
        assert abs((fp - fm) / (2 * h) - form.reshape(-1)[c]) < 1e-7 * max(1.0, abs(form.reshape(-1)[c]))


def test_seed_is_the_loss_gradient():
    """lambda(T) = 2 P^T P y is the gradient of the plane intensity in y."""
    sc = S.config_3d(n=6, fill=0.2)
    y = S.random_vector(sc.grid.nunk, 7)
    lam = adjoint.plane_adjoint_seed(sc.grid, y, sc.plane)
    d = S.random_vector(sc.grid.nunk, 8)
    h = 1e-6
    fd = (yee.intensity(sc.grid, y + h * d, sc.plane) - yee.intensity(sc.grid, y - h * d, sc.plane)) / (2 * h)
    assert abs(fd - lam @ d) < 1e-6 * abs(fd)
