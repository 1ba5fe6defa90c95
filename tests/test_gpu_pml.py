"""GPU parity of the paper's 2D PML model (auxiliary field P, eq. (mxw))
through the C ABI, against the oracle ``oracle.pml``: the operator and its
transpose element by element (FP64 1e-13, FP32 1e-6 relative L2 as for the
lossy-layer operator), responses by the plain method and by restart in
Krylov dimension against the exact solution (FP64 1e-10 / 1e-9), and the
descriptors the model does not accept."""
import ctypes

import numpy as np
import pytest

import scenario as S
from oracle import exact, pml

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

from paper_1707_00023_gb300 import Context, KxError  # noqa: E402
from paper_1707_00023_gb300 import _binding  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def dev(x, dtype):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda")


GRIDS = {
    "pec_pec": S.Grid(2, (37, 29), (S.PEC, S.PEC), 0, 5, 2.0, pml=1),
    "pec_periodic": S.Grid(2, (31, 20), (S.PEC, S.PERIODIC), 0, 4, 3.0, pml=1),
}


def eps_of(grid, seed=1):
    return 1.0 + 3.0 * np.random.default_rng(seed).random(grid.shape)


@pytest.mark.parametrize("name", list(GRIDS))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("transpose", [False, True])
def test_apply_A(name, prec, transpose):
    grid = GRIDS[name]
    eps = eps_of(grid)
    op = pml.PmlOperator(grid, eps)
    ctx = Context(grid, eps, precision=prec, krylov_dim=8)
    assert ctx.n == 4 * grid.ncell
    dt = torch.float64 if prec == "fp64" else torch.float32
    for seed in (2, 3):
        v = S.random_vector(grid.nunk, seed)           # wall entries non-zero: must be ignored
        w = ctx.apply_A(dev(v, dt), transpose=transpose).double().cpu().numpy()
        want = op.apply_T(v * S.wall_keep_mask(grid)) if transpose else op.apply(v)
        assert rel(w, want) < (1e-13 if prec == "fp64" else 1e-6)
    ctx.close()


def _plane_ez(grid, y, plane):
    nx, ny = grid.n
    Ez = y[2 * grid.ncell:3 * grid.ncell].reshape(ny, nx)
    return Ez[:, plane[1]] if plane[0] == 0 else Ez[plane[1], :]


def test_plain_response_fp64_against_exact():
    sc = S.config_2d_pml(n=24, ndisks=4, T=40.0)
    A = pml.PmlOperator(sc.grid, sc.eps_cell).matrix()
    oms = S.freq_list(2)
    ctx = Context(sc.grid, sc.eps_cell, precision="fp64", krylov_dim=30, max_freqs=2, batch=2)
    out = ctx.response_at_freqs(dev(sc.g, torch.float64), oms, sc.T, rtol=1e-11, method="plain", plane=sc.plane,
                                want_full=True)
    ctx.close()
    assert tuple(out["E_plane"].shape) == (2, 1, 24)
    for f, W in enumerate(oms):
        want = exact.y_plain(A, sc.g, W, sc.T)
        assert rel(out["Y"][f].cpu().numpy(), want) < 1e-10
        pe = _plane_ez(sc.grid, want, sc.plane)
        assert rel(out["E_plane"][f, 0].cpu().numpy(), pe) < 1e-10
        assert abs(out["intensity"][f] - (pe * pe).sum()) < 1e-9 * (pe * pe).sum()


def test_restart_in_dimension_fp64_against_exact():
    sc = S.config_2d_pml(n=24, ndisks=4, T=40.0)
    A = pml.PmlOperator(sc.grid, sc.eps_cell).matrix()
    oms = S.freq_list(3)
    ctx = Context(sc.grid, sc.eps_cell, precision="fp64", krylov_dim=32, max_freqs=3, batch=2, rst_samples=8000)
    out = ctx.response_restart_dim(dev(sc.g, torch.float64), oms, sc.T, rtol=1e-12, plane=sc.plane, want_full=True)
    ctx.close()
    for f, W in enumerate(oms):
        assert rel(out["Y"][f].cpu().numpy(), exact.y_plain(A, sc.g, W, sc.T)) < 1e-9


def test_descriptors_the_model_rejects():
    eps3 = np.ones((6, 6, 6))
    with pytest.raises(KxError, match="PML"):
        Context(S.Grid(3, (6, 6, 6), (0, 0, 1), 2, 1, 1.0, pml=1), eps3)
    g2 = S.Grid(2, (12, 12), (S.PEC, S.PEC), 1, 2, 1.0, pml=1)
    with pytest.raises(KxError, match="layer_axis 0"):
        Context(g2, np.ones(g2.shape))
    g2 = S.Grid(2, (12, 12), (S.PEC, S.PEC), 0, 2, 1.0, pml=1)
    with pytest.raises(KxError, match="adjoint"):
        Context(g2, np.ones(g2.shape), batch=2, max_checkpoints=4)
    # the allocation-free Arnoldi does not take the model either
    lib = _binding.load_library()
    d = _binding.Desc()
    d.dim, d.layer_axis, d.layer_cells, d.sigma_max = 2, 0, 2, 1.0
    d.n = (ctypes.c_int * 3)(12, 12, 1)
    d.bc = (ctypes.c_int * 3)(1, 1, 0)
    d.precision = _binding.KX_FP64
    d.pml = 1
    n = 4 * 144
    v0 = torch.ones(n, dtype=torch.float64, device="cuda")
    V = torch.zeros(n * 5, dtype=torch.float64, device="cuda")
    H = torch.zeros(5 * 4, dtype=torch.float64, device="cuda")
    eps = torch.ones(144, dtype=torch.float64, device="cuda")
    beta, md = ctypes.c_double(), ctypes.c_int()
    st = lib.kx_arnoldi_noalloc(ctypes.byref(d), ctypes.c_void_p(eps.data_ptr()), ctypes.c_void_p(v0.data_ptr()), 4,
                                ctypes.c_void_p(V.data_ptr()), ctypes.c_void_p(H.data_ptr()), ctypes.byref(beta),
                                ctypes.byref(md), None)
    assert st == _binding.KX_EINVAL and b"PML" in lib.kx_noalloc_last_error()
