"""The allocation-free Arnoldi entry point against the context-based one.

Callers that cannot allocate device memory (code inside another runtime's
memory pool or a captured graph, plug-ins with a fixed arena, services that
forbid cudaMalloc after start-up) use kx_arnoldi_noalloc, which keeps its
scratch in a fixed device array inside the library.  This test calls it
through the C ABI twice in a row, with different start vectors, and checks
each result against arnoldi() on a context, within the tolerances used for
arnoldi() in the parity tests.  The file is named to be collected last.
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


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_arnoldi_matches_context(prec):
    grid = S.Grid(3, (20, 18, 23), (S.PERIODIC, S.PERIODIC, S.PEC), 2, 3, 1.0)
    eps = 1.0 + 3.0 * np.random.default_rng(11).random(grid.shape)
    dt = torch.float64 if prec == "fp64" else torch.float32
    m = 12
    lib = _binding.load_library()
    ctx = Context(grid, eps, precision=prec, krylov_dim=16)
    d = _binding.Desc()
    ctypes.memmove(ctypes.byref(d), ctypes.byref(ctx.desc), ctypes.sizeof(d))
    eps_dev = torch.tensor(eps.reshape(-1), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for seed in (21, 22):
        v0 = torch.tensor(S.masked_random_vector(grid, seed), dtype=dt, device="cuda")
        V_ref, H_ref, b_ref, md_ref = ctx.arnoldi(v0, m)
        V = torch.empty((m + 1, grid.nunk), dtype=dt, device="cuda")
        H = torch.empty((m, m + 1), dtype=torch.float64, device="cuda")   # (m+1) x m column-major
        beta = ctypes.c_double()
        md = ctypes.c_int()
        st = lib.kx_arnoldi_noalloc(ctypes.byref(d), ctypes.c_void_p(eps_dev.data_ptr()),
                                    ctypes.c_void_p(v0.data_ptr()), m, ctypes.c_void_p(V.data_ptr()),
                                    ctypes.c_void_p(H.data_ptr()), ctypes.byref(beta), ctypes.byref(md),
                                    ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, lib.kx_noalloc_last_error().decode()
        assert md.value == md_ref == m
        Hn = H.cpu().numpy().T
        Vn = V.cpu().numpy()
        Vr = V_ref.cpu().numpy()
        if prec == "fp64":
            assert abs(beta.value - b_ref) < 1e-12 * b_ref
            assert np.abs(Hn - H_ref).max() < 1e-11 * np.abs(H_ref).max()
            assert np.abs(Vn - Vr).max() < 1e-10
        else:
            assert abs(beta.value - b_ref) < 1e-6 * b_ref
            assert np.abs(Hn - H_ref).max() < 1e-4 * np.abs(H_ref).max()
    # a Krylov dimension beyond the scratch array is refused with a message
    st = lib.kx_arnoldi_noalloc(ctypes.byref(d), ctypes.c_void_p(eps_dev.data_ptr()),
                                ctypes.c_void_p(v0.data_ptr()), 65, ctypes.c_void_p(V.data_ptr()),
                                ctypes.c_void_p(H.data_ptr()), ctypes.byref(beta), ctypes.byref(md),
                                ctypes.c_void_p(stream.cuda_stream))
    assert st == _binding.KX_EINVAL
    assert b"64" in lib.kx_noalloc_last_error()
    ctx.close()
