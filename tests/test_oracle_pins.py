"""Pins of the FP64 oracle against closed forms, invariants and brute force.

Each test fixes one piece of the oracle to something other than the oracle
itself (a closed-form spectrum, a conservation law, a geometric brute-force
definition, an identity of the paper), so that a dropped term, a wrong sign
or a shifted index fails at least one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

import scenario as S
from oracle import exact, krylov, yee

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def homogeneous(dim, n, eps=1.0, bc=None, sigma_max=0.0, layer=1, layer_axis=None):
    if bc is None:
        bc = (S.PERIODIC,) * dim
    if layer_axis is None:
        layer_axis = dim - 1 if dim == 3 else 0
    grid = S.Grid(dim, (n,) * dim, bc, layer_axis, layer, sigma_max)
    return grid, np.full(grid.shape, eps)


def plane_wave_block(op, kvec):
    """Restriction of A to the plane waves exp(i k . r_c) of each component.

    Homogeneous media make A translation invariant, so each single-component
    plane wave maps into the span of the plane waves of all components.
    """
    g = op.grid
    nc = g.ncomp
    basis = []
    for c in range(nc):
        coords = yee.node_coords(g, c)
        phase = sum(kvec[a] * coords[a] for a in range(g.dim))
        vec = np.zeros(g.nunk, np.complex128)
        vec[c * g.ncell:(c + 1) * g.ncell] = np.exp(1j * phase).reshape(-1)
        basis.append(vec)
    B = np.stack(basis, 1)
    AB = np.stack([op.apply(b.real) + 1j * op.apply(b.imag) for b in basis], 1)
    coef, *_ = np.linalg.lstsq(B, AB, rcond=None)
    assert np.linalg.norm(B @ coef - AB) < 1e-10 * max(1.0, np.linalg.norm(AB))
    return coef


@pytest.mark.parametrize("dim", [2, 3])
def test_plane_wave_dispersion(dim):
    """Yee semi-discrete dispersion: omega^2 = (1/eps) sum_d (2 sin(k_d/2))^2."""
    n = 8
    eps = 2.25
    grid, e = homogeneous(dim, n, eps)
    op = yee.Operator(grid, e)
    rng = np.random.default_rng(3)
    for _ in range(4):
        m = rng.integers(0, n, size=dim)
        k = 2 * np.pi * m / n
        omega = math.sqrt(sum((2 * math.sin(kk / 2)) ** 2 for kk in k) / eps)
        ev = np.linalg.eigvals(plane_wave_block(op, k))
        assert np.all(np.abs(ev.real) < 1e-12)
        got = np.sort(np.abs(ev.imag))
        if dim == 2:
            want = np.sort([0.0, omega, omega])
        else:
            want = np.sort([0.0, 0.0, omega, omega, omega, omega])
        np.testing.assert_allclose(got, want, atol=1e-12)


def test_plane_wave_time_evolution():
    """exp(-tA) on a plane-wave eigenvector is the phase rotation e^{-i omega t}."""
    grid, e = homogeneous(3, 6, 1.0)
    op = yee.Operator(grid, e)
    A = op.matrix()
    k = 2 * np.pi * np.array([1, 2, 0]) / 6
    blk = plane_wave_block(op, k)
    ev, W = np.linalg.eig(blk)
    i = int(np.argmax(ev.imag))
    lam = ev[i]
    omega = math.sqrt(sum((2 * math.sin(kk / 2)) ** 2 for kk in k))
    assert abs(lam - 1j * omega) < 1e-12
    u = np.zeros(grid.nunk, np.complex128)
    for c in range(grid.ncomp):
        coords = yee.node_coords(grid, c)
        ph = sum(k[a] * coords[a] for a in range(3))
        u[c * grid.ncell:(c + 1) * grid.ncell] = W[c, i] * np.exp(1j * ph).reshape(-1)
    t = 3.7
    got = spla.expm_multiply(-t * A, u.real)
    want = np.real(np.exp(-lam * t) * u)
    assert np.linalg.norm(got - want) < 1e-11 * np.linalg.norm(want)


def test_pec_cavity_spectrum_golden():
    """2D PEC cavity resonances equal the closed-form Dirichlet-Laplacian
    values stored in tests/golden/cavity_2d_n6.txt (pins the wall nodes)."""
    want = np.loadtxt(os.path.join(GOLDEN, "cavity_2d_n6.txt"))
    grid, e = homogeneous(2, 6, 1.0, bc=(S.PEC, S.PEC))
    op = yee.Operator(grid, e)
    keep = op.keep_vector().astype(bool)
    Ad = op.matrix().toarray()[np.ix_(keep, keep)]
    ev = np.linalg.eigvals(Ad)
    assert np.all(np.abs(ev.real) < 1e-10)
    pos = np.sort(ev.imag[ev.imag > 1e-8])
    np.testing.assert_allclose(pos, want, atol=1e-10)


def test_pec_slab_spectrum_3d():
    """3D grid periodic in x, y with PEC at z = 0 (= n): modes are Fourier in
    x, y and sine/cosine in z; omega^2 = kx'^2 + ky'^2 + (2 sin(p pi/2n))^2,
    twice for p = 1..n-1 and once (the E_z-H_x-H_y family) for p = 0."""
    n = 4
    grid, e = homogeneous(3, n, 1.0, bc=(S.PERIODIC, S.PERIODIC, S.PEC))
    op = yee.Operator(grid, e)
    keep = op.keep_vector().astype(bool)
    Ad = op.matrix().toarray()[np.ix_(keep, keep)]
    ev = np.linalg.eigvals(Ad)
    pos = np.sort(ev.imag[ev.imag > 1e-8])
    want = []
    for mx, my in itertools.product(range(n), range(n)):
        kx = 2 * math.sin(math.pi * mx / n)
        ky = 2 * math.sin(math.pi * my / n)
        for p in range(n):
            kz = 2 * math.sin(p * math.pi / (2 * n))
            w = math.sqrt(kx * kx + ky * ky + kz * kz)
            if w < 1e-12:
                continue
            want += [w, w] if p >= 1 else [w]
    np.testing.assert_allclose(pos, np.sort(want), atol=1e-10)


@pytest.mark.parametrize("cfg", ["2d", "3d"])
def test_skew_and_dissipation_structure(cfg):
    """M A - Sigma is exactly skew, and y^T M A y = y^T Sigma y: the damping
    enters the E rows as sigma/eps (matrix form of eq. (ode))."""
    sc = S.config_2d(n=10, ndisks=2) if cfg == "2d" else S.config_3d(n=6, fill=0.2)
    # permittivity varies inside the absorbing layer too, so sigma and eps overlap
    eps = 1.0 + np.random.default_rng(9).random(sc.grid.shape) * 3.0
    op = yee.Operator(sc.grid, eps)
    A = op.matrix().toarray()
    M = op.weights()
    P = op.keep_vector()
    C = M[:, None] * A - np.diag(op.sigma_vector() * P)
    assert np.abs(C + C.T).max() < 1e-14
    y = S.masked_random_vector(sc.grid, 5)
    lhs = y @ (M * op.apply(y))
    rhs = y @ (op.sigma_vector() * y)
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)
    assert rhs > 0


@pytest.mark.parametrize("cfg", ["2d", "3d"])
def test_stencil_matches_block_matrix(cfg):
    """Component formulas of eq. (mxw) = block matrix of eq. (ode), and the
    transpose action = the transposed matrix."""
    sc = S.config_2d(n=12, ndisks=3) if cfg == "2d" else S.config_3d(n=8, fill=0.25)
    op = yee.Operator(sc.grid, sc.eps_cell)
    A = op.matrix()
    v = S.random_vector(sc.grid.nunk, 11)
    np.testing.assert_allclose(op.apply(v), A @ v, atol=1e-13)
    np.testing.assert_allclose(op.apply_T(v), A.T @ v, atol=1e-13)


def test_energy_conserved_without_damping():
    """sigma = 0: y^T M y is constant along exp(-tA) y0 (A skew in the M inner
    product)."""
    sc = S.config_3d(n=8, fill=0.3)
    grid = S.Grid(3, sc.grid.n, sc.grid.bc, 2, sc.grid.layer_cells, 0.0)
    op = yee.Operator(grid, sc.eps_cell)
    A = op.matrix()
    M = op.weights()
    y0 = S.masked_random_vector(grid, 2)
    e0 = y0 @ (M * y0)
    y = spla.expm_multiply(-4.0 * A, y0)
    assert abs(y @ (M * y) - e0) < 1e-12 * e0


def test_energy_decays_with_damping():
    """sigma > 0: the M-norm of exp(-tA) y0 is non-increasing (the transient
    y^ of eq. (y_homo) decays)."""
    sc = S.config_2d(n=16, ndisks=3)
    op = yee.Operator(sc.grid, sc.eps_cell)
    A = op.matrix()
    M = op.weights()
    y = S.masked_random_vector(sc.grid, 4)
    prev = y @ (M * y)
    for _ in range(6):
        y = spla.expm_multiply(-2.0 * A, y)
        cur = y @ (M * y)
        assert cur <= prev * (1 + 1e-13)
        prev = cur
    assert prev < 0.9 * (S.masked_random_vector(sc.grid, 4) @ (M * S.masked_random_vector(sc.grid, 4)))


def test_eps_average_brute_force():
    """eps on each E node = mean over the cells whose closure holds the node,
    found by brute-force geometry over all cells."""
    for dim in (2, 3):
        n = 4
        grid = S.Grid(dim, (n,) * dim, (S.PERIODIC,) * dim, 0, 1, 0.0)
        rng = np.random.default_rng(7)
        eps_cell = 1.0 + rng.random(grid.shape)
        op = yee.Operator(grid, eps_cell)
        nh = 2 if dim == 2 else 3
        for c in range(nh, grid.ncomp):
            coords = yee.node_coords(grid, c)
            got = op.eps[c]
            for idx in itertools.product(*[range(n)] * dim):
                p = [coords[a][idx] for a in range(dim)]   # idx is slowest-first
                vals = []
                for cell in itertools.product(*[range(n)] * dim):   # (x, y[, z])
                    inside = True
                    for a in range(dim):
                        d = (p[a] - cell[a]) % n
                        if not (d <= 1.0 + 1e-12 or d >= n - 1e-12):
                            inside = False
                    if inside:
                        vals.append(eps_cell[tuple(reversed(cell))])
                assert len(vals) == 4
                assert abs(got[idx] - np.mean(vals)) < 1e-15


def test_sigma_profile_values():
    """Linear ramp: sigma_max at the wall, sigma_max/2 at half depth, 0 from
    the layer's inner edge on, on the node's own staggered coordinate."""
    grid = S.Grid(3, (16, 16, 16), (S.PERIODIC, S.PERIODIC, S.PEC), 2, 4, 2.0)
    sx = yee.sigma_nodes(grid, 3)      # Ex: integer z
    sz = yee.sigma_nodes(grid, 5)      # Ez: z + 1/2
    assert sx[0, 0, 0] == 2.0 and sx[2, 0, 0] == 1.0 and sx[4, 0, 0] == 0.0
    assert sx[8, 3, 5] == 0.0 and sx[14, 0, 0] == 1.0
    assert abs(sz[0, 0, 0] - 2.0 * 3.5 / 4) < 1e-15
    assert abs(sz[15, 0, 0] - 2.0 * 3.5 / 4) < 1e-15
    assert sz[4, 0, 0] == 0.0


@pytest.mark.parametrize("cfg", ["2d", "3d"])
def test_split_equals_plain(cfg):
    """Eq. (split1): Im(e^{i w T} z) - exp(-TA) Im z equals the solution of
    eq. (ode) computed by the augmented route, and both satisfy the ODE."""
    sc = S.config_2d(n=12, ndisks=2) if cfg == "2d" else S.config_3d(n=8, fill=0.2)
    op = yee.Operator(sc.grid, sc.eps_cell)
    A = op.matrix()
    om = 1.3 * S.OMEGA0
    T = 7.5
    y1 = exact.y_plain(A, sc.g, om, T)
    y2 = exact.y_split(A, sc.g, om, T)
    assert np.linalg.norm(y1 - y2) < 1e-12 * np.linalg.norm(y1)
    # ODE residual by central differences in T: y' = -A y + sin(wT) g
    h = 1e-3
    yp = (exact.y_split(A, sc.g, om, T + h) - exact.y_split(A, sc.g, om, T - h)) / (2 * h)
    res = yp + A @ y2 - math.sin(om * T) * sc.g
    assert np.linalg.norm(res) < 1e-5 * np.linalg.norm(yp)
    # y(0) = 0 and the small-t limit y(t) ~ (1 - cos wt)/w g
    t = 1e-4
    ys = exact.y_plain(A, sc.g, om, t)
    np.testing.assert_allclose(ys, (1 - math.cos(om * t)) / om * sc.g, atol=1e-12)


def test_stationary_part():
    """z = (A + i w I)^{-1} g satisfies its time-harmonic equation to 1e-10
    (residual taken with the stencil, not the factorised matrix)."""
    sc = S.config_2d(n=16, ndisks=3)
    op = yee.Operator(sc.grid, sc.eps_cell)
    A = op.matrix()
    for om in (0.8 * S.OMEGA0, S.OMEGA0, 1.2 * S.OMEGA0):
        z = exact.z_stat(A, sc.g, om)
        assert exact.stationary_residual(op.apply, sc.g, om, z) < 1e-10


def test_arnoldi_relations():
    """Eqs. (Arn), (Krylov), (Arn1): A V_m = V_{m+1} H, V orthonormal,
    v_1 = g/||g||, H upper Hessenberg, span = K_m(A, g)."""
    sc = S.config_2d(n=12, ndisks=2)
    op = yee.Operator(sc.grid, sc.eps_cell)
    A = op.matrix()
    m = 12
    V, H, beta, md = krylov.arnoldi(op.apply, sc.g, m)
    assert md == m
    np.testing.assert_allclose(A @ V[:, :m], V @ H, atol=1e-13)
    np.testing.assert_allclose(V.T @ V, np.eye(m + 1), atol=1e-12)
    np.testing.assert_allclose(V[:, 0] * beta, sc.g, atol=1e-15)
    assert np.all(np.tril(H, -2) == 0)
    # Krylov span: the power basis lies in span(V)
    Kp = [sc.g / np.linalg.norm(sc.g)]
    for _ in range(m - 1):
        w = A @ Kp[-1]
        Kp.append(w / np.linalg.norm(w))
    Kp = np.stack(Kp, 1)
    resid = Kp - V[:, :m] @ (V[:, :m].T @ Kp)
    assert np.linalg.norm(resid) < 1e-8


def test_lemma1_residual():
    """Lemma 1: the explicit residual -A y_m - y_m' + sin(wt) g of the Krylov
    approximation y_m = V_m u(t) (u from eq. (corr2)) equals
    -h_{m+1,m} (e_m^T u) v_{m+1}; y_m' by central differences of u."""
    sc = S.config_2d(n=12, ndisks=2)
    op = yee.Operator(sc.grid, sc.eps_cell)
    m = 4
    V, H, beta, _ = krylov.arnoldi(op.apply, sc.g, m)
    om = S.OMEGA0
    for t in (2.5, 6.0):
        u = krylov.proj_sine(H, beta, om, t)
        d = 1e-3
        du = (krylov.proj_sine(H, beta, om, t + d) - krylov.proj_sine(H, beta, om, t - d)) / (2 * d)
        ym = V[:, :m] @ u
        r_explicit = -op.apply(ym) - V[:, :m] @ du + math.sin(om * t) * sc.g
        r_formula = krylov.lemma1_residual(H, u, V[:, m])
        assert np.linalg.norm(r_formula) > 1e-2 * np.linalg.norm(sc.g)
        assert np.linalg.norm(r_explicit - r_formula) < 1e-6 * np.linalg.norm(r_formula)


def test_corollary1_one_basis_all_frequencies():
    """Corollary 1: one Krylov basis of K_m(A, g) serves every frequency;
    only the projected problem changes.  Unrestarted, large m, short T."""
    sc = S.config_2d(n=10, ndisks=2)
    op = yee.Operator(sc.grid, sc.eps_cell)
    A = op.matrix()
    T = 3.0
    V, H, beta, md = krylov.arnoldi(op.apply, sc.g, 60)
    for om in S.freq_list(3):
        want = exact.y_plain(A, sc.g, om, T)
        u1 = krylov.proj_sine(H, beta, om, T)
        u2 = krylov.proj_sine_phi(H, beta, om, T)
        assert np.linalg.norm(V[:, :md] @ u1 - want) < 1e-10 * np.linalg.norm(want)
        assert np.linalg.norm(u1 - u2) < 1e-12 * np.linalg.norm(u1)


def test_projected_closed_forms():
    """exp(-tau H) beta e1 for a rotation, a diagonal and a nilpotent H, and
    phi_1 for a diagonal argument."""
    om, tau = 0.7, 2.3
    R = np.array([[0.0, -om], [om, 0.0], [0.0, 0.0]])
    np.testing.assert_allclose(krylov.proj_exp(R, tau, 2.0),
                               2.0 * np.array([math.cos(om * tau), -math.sin(om * tau)]), atol=1e-14)
    d = np.array([0.5, 1.0, 3.0])
    D = np.vstack([np.diag(d), np.zeros((1, 3))])
    np.testing.assert_allclose(krylov.proj_exp(D, tau, 1.0), [math.exp(-0.5 * tau), 0, 0], atol=1e-15)
    m = 5
    Nm = np.zeros((m + 1, m))
    for k in range(m - 1):
        Nm[k + 1, k] = -1.0       # H = -N, N e_k = e_{k+1}
    want = np.array([tau ** k / math.factorial(k) for k in range(m)])
    np.testing.assert_allclose(krylov.proj_exp(Nm, tau, 1.0), want, rtol=1e-13)
    X = np.diag([-1.0, -0.2, 0.5]).astype(complex)
    b = np.array([1.0, 2.0, 3.0], complex)
    want = (np.exp(np.diag(X)) - 1) / np.diag(X) * b
    np.testing.assert_allclose(krylov.phi1_times(X, b), want, rtol=1e-13)


def test_proj_sine_scalar_closed_form():
    """m = 1: u' = -h u + beta sin(wt), u(0) = 0 has the closed form
    beta (h sin wt - w cos wt + w e^{-ht}) / (h^2 + w^2)."""
    h, beta, om, T = 0.3, 1.7, 0.9, 4.1
    H = np.array([[h], [0.0]])
    want = beta * (h * math.sin(om * T) - om * math.cos(om * T) + om * math.exp(-h * T)) / (h * h + om * om)
    assert abs(krylov.proj_sine(H, beta, om, T)[0] - want) < 1e-13 * abs(want)
    assert abs(krylov.proj_sine_phi(H, beta, om, T)[0] - want) < 1e-13 * abs(want)


def test_shifted_fom_reaches_stationary_solution():
    """Restarted shifted FOM on one shared basis converges to the sparse-LU
    z_stat for every shift."""
    sc = S.config_2d(n=10, ndisks=2)
    op = yee.Operator(sc.grid, sc.eps_cell)
    A = op.matrix()
    oms = S.freq_list(4)
    z, rel, cycles = krylov.shifted_fom(op.apply, sc.g, oms, 40, 1e-11)
    assert np.all(rel < 1e-11)
    for j, om in enumerate(oms):
        zz = exact.z_stat(A, sc.g, om)
        assert np.linalg.norm(z[j] - zz) < 1e-8 * np.linalg.norm(zz)


def test_plane_extraction_and_intensity():
    sc = S.config_3d(n=8, fill=0.2)
    g = sc.grid
    y = np.arange(g.nunk, dtype=float)
    P = yee.plane_fields(g, y, (2, 5))
    nc = g.ncell
    for q in range(3):
        comp = y[(3 + q) * nc:(4 + q) * nc].reshape(8, 8, 8)
        np.testing.assert_array_equal(P[q], comp[5].reshape(-1))
    assert yee.intensity(g, y, (2, 5)) == float((P * P).sum())


def test_plain_route_by_pieces():
    """The augmented route taken one sub-interval at a time (the semigroup
    property exp((s + t) L) = exp(s L) exp(t L)): its intermediate states are
    the split1 solution at those times (eq. (split1), an independent route),
    and a different balance eta of the phase entries gives the same y."""
    sc = S.config_3d(n=8, fill=0.2)
    A = yee.Operator(sc.grid, sc.eps_cell).matrix()
    om = 0.9 * S.OMEGA0
    T = 6.0
    states = list(exact.y_plain_pieces(A, sc.g, om, T, 4, eta=float(np.abs(sc.g).sum())))
    assert [k for k, _ in states] == [1, 2, 3, 4]
    for k, y in states:
        want = exact.y_split(A, sc.g, om, k * T / 4)
        assert np.linalg.norm(y - want) < 1e-11 * np.linalg.norm(want)
