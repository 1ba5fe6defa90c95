"""Pins of the restart-in-dimension oracle (Sect. 3.4, eq. (rst),
Corollary 2, Fig. alg:rst) against facts fixed outside it: the exact
solution of eq. (ode), the residual of the restarted iterate computed from
the operator itself, the basis' independence of the frequency, and the exact
answer once the Krylov space is invariant."""
import numpy as np
import pytest

import scenario as S
from oracle import exact, krylov, restart, yee


def _case(cfg):
    """A small scenario with a random source (a plane source on a nearly
    uniform periodic grid spans too few Krylov directions to need restarts)."""
    if cfg == "2d":
        sc = S.config_2d(n=10, ndisks=2)
        m = 12
    else:
        sc = S.config_3d(n=8, fill=0.25)
        m = 16
    sc.g = S.masked_random_vector(sc.grid, 77)
    return sc, 30.0, m


@pytest.mark.parametrize("cfg", ["2d", "3d"])
def test_converges_to_exact_solution(cfg):
    """Restarted to convergence, every frequency's y(T) is the exact
    solution of y' = -A y + sin(W t) g (matrix exponential of the augmented
    system, a library routine independent of the Krylov code)."""
    sc, T, m = _case(cfg)
    op = yee.Operator(sc.grid, sc.eps_cell)
    A = op.matrix()
    oms = [0.8, 1.0, 1.2]
    out = restart.restart_dim(op.apply, sc.g, oms, T, m, max_restarts=60, rtol=1e-13)
    assert all(out["converged"])
    assert min(out["restarts"]) >= 3, "the case must exercise several restarts"
    for f, W in enumerate(oms):
        ref = exact.y_plain(A, sc.g, W, T)
        assert np.linalg.norm(out["y"][f] - ref) <= 1e-9 * np.linalg.norm(ref)


def test_first_restart_is_the_unrestarted_method():
    """With one restart the iterate is V_m u(T), u from eq. (corr2) with
    alpha = sin(W t) (the m+2 augmented exponential of the unrestarted
    method)."""
    sc, T, m = _case("2d")
    op = yee.Operator(sc.grid, sc.eps_cell)
    W = 1.1
    out = restart.restart_dim(op.apply, sc.g, [W], T, m, max_restarts=1, rtol=0.0)
    V, H, beta, md = krylov.arnoldi(op.apply, sc.g, m)
    y1 = V[:, :md] @ krylov.proj_sine(H, beta, W, T)
    assert np.linalg.norm(out["y"][0] - y1) <= 1e-12 * np.linalg.norm(y1)


@pytest.mark.parametrize("K", [1, 3])
def test_residual_is_alphahat_times_v_next(K):
    """eq. (resid) after K restarts: sin(W t) g - y'(t) - A y(t) equals
    alphahat_{K+1}(t) v_{m+1}.  y' comes from central differences of the
    iterate and A y from the operator, so a wrong sign, index or scale in the
    restart coupling shows up here."""
    sc, T, m = _case("3d")
    op = yee.Operator(sc.grid, sc.eps_cell)
    W = 0.95
    t0, dl = 11.3, 1e-3
    out = restart.restart_dim(op.apply, sc.g, [W], T, m, max_restarts=K, rtol=0.0,
                              t_eval=(t0 - dl, t0, t0 + dl))
    ym, y0, yp = out["y_t"][0]
    dy = (yp - ym) / (2 * dl)
    r = np.sin(W * t0) * sc.g - dy - op.apply(y0)
    pred = restart.alpha_at(out["alpha"][0], t0) * out["v_next"]
    scale = np.linalg.norm(sc.g)
    assert np.linalg.norm(pred) > 1e-3 * scale, "the residual must be far from zero for the pin to bite"
    assert np.linalg.norm(r - pred) <= 1e-5 * scale


def test_one_basis_serves_every_frequency():
    """Corollary 2: frequencies solved together equal each solved alone."""
    sc, T, m = _case("2d")
    op = yee.Operator(sc.grid, sc.eps_cell)
    oms = [0.85, 1.15]
    joint = restart.restart_dim(op.apply, sc.g, oms, T, m, max_restarts=4, rtol=0.0)
    for f, W in enumerate(oms):
        alone = restart.restart_dim(op.apply, sc.g, [W], T, m, max_restarts=4, rtol=0.0)
        assert np.array_equal(joint["y"][f], alone["y"][0])


def test_invariant_subspace_gives_the_exact_answer():
    """With m at least the dimension of the Krylov space, the Arnoldi
    process breaks down, the projection is exact and one restart suffices."""
    grid = S.Grid(2, (4, 3), (S.PEC, S.PEC), 0, 1, 0.5)
    rng = np.random.default_rng(3)
    eps = 1.0 + rng.random(grid.shape)
    op = yee.Operator(grid, eps)
    g = S.masked_random_vector(grid, 5)
    out = restart.restart_dim(op.apply, g, [1.0], 7.0, grid.nunk + 2, max_restarts=5, rtol=1e-12)
    assert out["restarts"][0] == 1 and out["converged"][0]
    ref = exact.y_plain(op.matrix(), g, 1.0, 7.0)
    assert np.linalg.norm(out["y"][0] - ref) <= 1e-9 * np.linalg.norm(ref)


def test_zero_source():
    sc, T, m = _case("2d")
    op = yee.Operator(sc.grid, sc.eps_cell)
    out = restart.restart_dim(op.apply, np.zeros_like(sc.g), [1.0], T, m)
    assert out["converged"][0] and not np.any(out["y"][0])


def test_sampled_residual_bounds_the_error():
    """The stopping test reads max_t |alphahat(t)|.  The error of the
    restarted iterate solves e' = -A e + alphahat(t) v_{m+1}, e(0) = 0, and
    exp(-sA) is a contraction in the energy norm ||x||_M (M = diag(1 on H,
    eps on E)), so ||e(T)||_2 <= sqrt(max M / min M) * T * max_t |alphahat|."""
    sc, T, m = _case("3d")
    op = yee.Operator(sc.grid, sc.eps_cell)
    A = op.matrix()
    W = 1.05
    out = restart.restart_dim(op.apply, sc.g, [W], T, m, max_restarts=3, rtol=0.0, nsample=2000)
    ref = exact.y_plain(A, sc.g, W, T)
    err = np.linalg.norm(out["y"][0] - ref)
    w = op.weights()
    kappa = np.sqrt(w.max() / w.min())
    assert 0.0 < err <= 1.01 * kappa * T * out["resid"][0]
