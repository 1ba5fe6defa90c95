"""GPU parity of the single-sweep Arnoldi form (descriptor arnoldi_form
KX_ARN_SWEEP; Sect. 3.2, eqs. (Arn), (Arn1)) through the C ABI.

In exact arithmetic it is classical Gram-Schmidt, so it is checked against
the oracle's Arnoldi process element by element: H and V in FP64 (1e-11 /
1e-10, as the two-pass form), the Arnoldi relation A V_m = V_{m+1} H with
the oracle operator, and orthogonality of V, on ragged 2D, 3D and PML grids,
for a few steps and for the largest Krylov dimension (64); grids with
nx % 4 == 0 run the FP32 quad kernels.  FP32 is held to the two-pass form's
bounds.  Restart-in-dimension responses with either form agree within the
precision's tolerance, and the single-sweep form launches two kernels per
step."""
import numpy as np
import pytest

import scenario as S
from oracle import exact, krylov, pml, yee

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

from paper_1707_00023_gb300 import Context  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def dev(x, dtype):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda")


GRIDS = {
    "2d_pec": S.Grid(2, (37, 29), (S.PEC, S.PEC), 0, 4, 1.0),
    "3d_pecz": S.Grid(3, (21, 18, 23), (S.PERIODIC, S.PERIODIC, S.PEC), 2, 3, 1.0),
    "3d_mixed": S.Grid(3, (16, 12, 10), (S.PEC, S.PERIODIC, S.PERIODIC), 0, 2, 0.5),
    "2d_pml": S.Grid(2, (31, 20), (S.PEC, S.PERIODIC), 0, 4, 3.0, pml=1),
    # nx % 4 == 0: the FP32 quad kernels (ragged y and z extents)
    "3d_quad": S.Grid(3, (20, 13, 11), (S.PEC, S.PERIODIC, S.PEC), 2, 2, 1.0),
}


def operator(grid, eps):
    return pml.PmlOperator(grid, eps) if getattr(grid, "pml", 0) else yee.Operator(grid, eps)


def eps_of(grid, seed=4):
    return 1.0 + 3.0 * np.random.default_rng(seed).random(grid.shape)


@pytest.mark.parametrize("name", list(GRIDS))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("m", [10, 64])
def test_sweep_arnoldi_matches_oracle(name, prec, m):
    grid = GRIDS[name]
    eps = eps_of(grid)
    op = operator(grid, eps)
    ctx = Context(grid, eps, precision=prec, krylov_dim=64, arnoldi="sweep")
    dt = torch.float64 if prec == "fp64" else torch.float32
    v0 = S.masked_random_vector(grid, 5)
    V, H, beta, md = ctx.arnoldi(dev(v0, dt), m)
    Vo, Ho, bo, mo = krylov.arnoldi(op.apply, v0, m)
    ctx.close()
    assert md == m == mo
    Vn = V.double().cpu().numpy().T
    AV = np.stack([op.apply(Vn[:, i]) for i in range(m)], 1)
    orth = np.abs(Vn.T @ Vn - np.eye(m + 1)).max()
    if prec == "fp64":
        assert abs(beta - bo) < 1e-12 * bo
        assert np.abs(H - Ho).max() < 1e-11 * np.abs(Ho).max()
        assert np.abs(Vn - Vo).max() < 1e-10
        assert np.linalg.norm(AV - Vn @ H) < 1e-12 * np.linalg.norm(AV)
        assert orth < 1e-12
    else:
        assert abs(beta - bo) < 1e-6 * bo
        # the first columns of H agree to FP32 rounding; later ones follow
        # the FP32 basis (as the two-pass form's)
        assert np.abs(H[:, :10] - Ho[:, :10]).max() < 1e-4 * np.abs(Ho).max()
        assert np.linalg.norm(AV - Vn @ H) < 2e-6 * np.linalg.norm(AV)
        assert orth < 2e-5


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sweep_matches_two_pass(prec):
    """The two forms on one 3D grid at m = 64: the same process up to rounding."""
    grid = GRIDS["3d_pecz"]
    eps = eps_of(grid, 7)
    dt = torch.float64 if prec == "fp64" else torch.float32
    v0 = dev(S.masked_random_vector(grid, 8), dt)
    out = {}
    for form in ("twopass", "sweep"):
        ctx = Context(grid, eps, precision=prec, krylov_dim=64, arnoldi=form)
        V, H, beta, md = ctx.arnoldi(v0, 64)
        out[form] = (V.double().cpu().numpy(), H, beta, md)
        ctx.close()
    (V1, H1, b1, m1), (V2, H2, b2, m2) = out["twopass"], out["sweep"]
    assert m1 == m2 == 64
    assert b1 == b2                        # the same norm kernel
    if prec == "fp64":
        assert np.abs(H1 - H2).max() < 1e-11 * np.abs(H1).max()
        assert np.abs(V1 - V2).max() < 1e-10
    else:
        assert np.abs(H1[:, :10] - H2[:, :10]).max() < 1e-4 * np.abs(H1).max()


def test_sweep_breakdown_invariant_subspace():
    """A plane wave of a homogeneous, lossless, periodic grid spans an
    invariant subspace of A of dimension 2: the sweep stops after 2 steps."""
    grid = S.Grid(3, (8, 8, 8), (S.PERIODIC,) * 3, 2, 1, 0.0)
    eps = np.full(grid.shape, 2.25)
    op = yee.Operator(grid, eps)
    k = 2 * np.pi / 8
    v = np.zeros(grid.nunk)
    coords = yee.node_coords(grid, 4)
    v[4 * grid.ncell:5 * grid.ncell] = np.cos(k * coords[0]).reshape(-1)
    ctx = Context(grid, eps, precision="fp64", krylov_dim=8, arnoldi="sweep")
    V, H, beta, md = ctx.arnoldi(dev(v, torch.float64), 6)
    ctx.close()
    Vo, Ho, _, mo = krylov.arnoldi(op.apply, v, 6)
    assert md == mo == 2
    assert np.abs(H[:3, :2] - Ho[:3, :2]).max() < 1e-12


def test_sweep_launches_two_kernels_a_step():
    grid = GRIDS["3d_mixed"]
    eps = eps_of(grid)
    ctx = Context(grid, eps, precision="fp32", krylov_dim=32, arnoldi="sweep")
    v0 = dev(S.masked_random_vector(grid, 3), torch.float32)
    ctx.arnoldi(v0, 32)                      # warm the grid caches
    ctx.reset_stats()
    ctx.set_timing(True)
    ctx.arnoldi(v0, 32)
    kt = ctx.kernel_times()
    ctx.set_timing(False)
    ctx.close()
    assert kt["sweep"]["launches"] == 32
    assert kt["swapply"]["launches"] == 33   # 32 apply passes and the closing finalisation
    assert kt["pass_a"]["launches"] == 0 and kt["pass_b"]["launches"] == 0


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-6)])
@pytest.mark.parametrize("nx", [14, 16])
def test_restart_dim_forms_agree(prec, tol, nx):
    """Restart in Krylov dimension with either form, against the exact
    solution and against each other (nx = 16: the FP32 quad kernels)."""
    grid = S.Grid(3, (nx, 11, 13), (S.PERIODIC, S.PERIODIC, S.PEC), 2, 2, 1.0)
    eps = eps_of(grid, 11)
    # a random source in the range of A (no curl-free part, see test_gpu_rstdim)
    g = yee.Operator(grid, eps).apply(S.masked_random_vector(grid, 12))
    oms = S.freq_list(3)
    T = 20.0
    dt = torch.float64 if prec == "fp64" else torch.float32
    Y = {}
    for form in ("twopass", "sweep"):
        ctx = Context(grid, eps, precision=prec, krylov_dim=24, max_freqs=3, batch=2, rst_samples=8000,
                      arnoldi=form)
        out = ctx.response_restart_dim(dev(g, dt), oms, T, rtol=1e-11 if prec == "fp64" else 1e-7, plane=(2, 9),
                                       want_full=True)
        Y[form] = out["Y"].double().cpu().numpy()
        ctx.close()
    A = yee.Operator(grid, eps).matrix()
    for f, W in enumerate(oms):
        want = exact.y_plain(A, g, W, T)
        assert rel(Y["sweep"][f], want) < (1e-9 if prec == "fp64" else 1e-6)
        assert rel(Y["sweep"][f], Y["twopass"][f]) < tol


def test_bounded_wait_runs_out_and_the_context_stays_usable():
    """The failure path of the sweep's bounded mbarrier waits, without a
    fault: a wait on a barrier that nothing completes runs out, the kernel
    reports KX_ETIMEOUT and returns, and the context then computes as before."""
    from paper_1707_00023_gb300 import _binding
    grid = GRIDS["3d_quad"]
    eps = eps_of(grid)
    op = yee.Operator(grid, eps)
    ctx = Context(grid, eps, precision="fp32", krylov_dim=16, arnoldi="sweep")
    assert ctx.wait_selftest(1000) == _binding.KX_ETIMEOUT
    assert b"ran out" in ctx.lib.kx_last_error(ctx.h)
    v = S.masked_random_vector(grid, 9)
    w = ctx.apply_A(dev(v, torch.float32)).double().cpu().numpy()
    assert rel(w, op.apply(v)) < 1e-6
    V, H, beta, md = ctx.arnoldi(dev(v, torch.float32), 16)
    Vo, Ho, _, _ = krylov.arnoldi(op.apply, v, 16)
    assert md == 16 and np.abs(H[:, :10] - Ho[:, :10]).max() < 1e-4 * np.abs(Ho).max()
    ctx.close()
