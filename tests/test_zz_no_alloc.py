"""The allocation-free Arnoldi entry point against the context-based one.

Callers that cannot allocate device memory (code inside another runtime's
memory pool, plug-ins with a fixed arena, services that forbid cudaMalloc
after start-up) use kx_arnoldi_noalloc, which keeps its scratch in a fixed
device array inside the library.  This test calls it through the C ABI twice
in a row, with different start vectors, and checks each result against
arnoldi() on a context, within the tolerances used for arnoldi() in the
parity tests; then at the largest Krylov dimension the array holds (m = 64),
and with a zero start vector, which is refused before any step.  The file is
named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import scenario as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

from paper_1707_00023_gb300 import Context, _binding  # noqa: E402


def _call(lib, d, eps_dev, v0, m, V, H, stream):
    beta = ctypes.c_double()
    md = ctypes.c_int()
    st = lib.kx_arnoldi_noalloc(ctypes.byref(d), ctypes.c_void_p(eps_dev.data_ptr()),
                                ctypes.c_void_p(v0.data_ptr()), m, ctypes.c_void_p(V.data_ptr()),
                                ctypes.c_void_p(H.data_ptr()), ctypes.byref(beta), ctypes.byref(md),
                                ctypes.c_void_p(stream.cuda_stream))
    return st, beta.value, md.value


def _check(prec, grid, eps, m, seeds):
    dt = torch.float64 if prec == "fp64" else torch.float32
    lib = _binding.load_library()
    ctx = Context(grid, eps, precision=prec, krylov_dim=m)
    d = _binding.Desc()
    ctypes.memmove(ctypes.byref(d), ctypes.byref(ctx.desc), ctypes.sizeof(d))
    eps_dev = torch.tensor(eps.reshape(-1), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    V = torch.empty((m + 1, grid.nunk), dtype=dt, device="cuda")
    H = torch.empty((m, m + 1), dtype=torch.float64, device="cuda")   # (m+1) x m column-major
    for seed in seeds:
        v0 = torch.tensor(S.masked_random_vector(grid, seed), dtype=dt, device="cuda")
        V_ref, H_ref, b_ref, md_ref = ctx.arnoldi(v0, m)
        st, beta, md = _call(lib, d, eps_dev, v0, m, V, H, stream)
        assert st == 0, lib.kx_noalloc_last_error().decode()
        assert md == md_ref == m
        Hn = H.cpu().numpy().T
        Vn = V.cpu().numpy()
        Vr = V_ref.cpu().numpy()
        if prec == "fp64":
            assert abs(beta - b_ref) < 1e-12 * b_ref
            assert np.abs(Hn - H_ref).max() < 1e-11 * np.abs(H_ref).max()
            assert np.abs(Vn - Vr).max() < 1e-10
        else:
            assert abs(beta - b_ref) < 1e-6 * b_ref
            assert np.abs(Hn - H_ref).max() < 1e-4 * np.abs(H_ref).max()
            assert np.abs(Vn - Vr).max() < 1e-5
    ctx.close()
    return lib, d, eps_dev, V, H, stream


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_arnoldi_matches_context(prec):
    grid = S.Grid(3, (20, 18, 23), (S.PERIODIC, S.PERIODIC, S.PEC), 2, 3, 1.0)
    eps = 1.0 + 3.0 * np.random.default_rng(11).random(grid.shape)
    m = 12
    lib, d, eps_dev, V, H, stream = _check(prec, grid, eps, m, (21, 22))
    dt = V.dtype
    # a Krylov dimension beyond the scratch array is refused with a message
    v0 = torch.tensor(S.masked_random_vector(grid, 23), dtype=dt, device="cuda")
    st, _, _ = _call(lib, d, eps_dev, v0, 65, V, H, stream)
    assert st == _binding.KX_EINVAL
    assert b"64" in lib.kx_noalloc_last_error()
    # a zero start vector is refused before any Arnoldi step, with its own message
    st, _, _ = _call(lib, d, eps_dev, torch.zeros_like(v0), m, V, H, stream)
    assert st == _binding.KX_ENONFINITE
    assert b"zero" in lib.kx_noalloc_last_error()
    # the entry point still works after the refusals
    st, beta, md = _call(lib, d, eps_dev, v0, m, V, H, stream)
    assert st == 0 and md == m and beta > 0


def test_noalloc_arnoldi_full_dimension():
    """m = 64, the most columns the scratch array holds, on a 3D grid of
    67k cells (FP64, compared with the context's arnoldi())."""
    grid = S.Grid(3, (44, 40, 38), (S.PERIODIC, S.PERIODIC, S.PEC), 2, 4, 1.0)
    eps = 1.0 + 1.25 * (np.random.default_rng(5).random(grid.shape) < 0.3)
    _check("fp64", grid, eps, 64, (31, 32))
