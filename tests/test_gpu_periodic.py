"""GPU parity of the periodic-source methods of Sect. 3.5 through the C ABI:
source splitting (eq. (split2), method "split2") and the neighbouring-
frequency difference of Fig. alg:spl1 (eq. (4diff), method "split4d").

Both reach the exact solution of eq. (ode) up to the Krylov tolerance, so
they are held to the same bars as the other responses: FP64 1e-10 relative
L2 against the oracle, FP32 1e-6 (split2, a chain of time-restarted
homogeneous solves like the plain method's).
"""
import numpy as np
import pytest

import scenario as S
from oracle import exact, periodic, yee

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

from paper_1707_00023_gb300 import Context  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def dev(x, dtype):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda")


def test_split2_fp64_matches_oracle():
    """T = 37 is not a whole number of periods: the remainder subinterval
    (its own w2) is exercised; two frequencies with different periods share
    the lockstep batch."""
    sc = S.config_2d(n=12, ndisks=2, T=37.0)
    op = yee.Operator(sc.grid, sc.eps_cell)
    A = op.matrix()
    oms = [1.07, 0.83]
    ctx = Context(sc.grid, sc.eps_cell, precision="fp64", krylov_dim=30, max_freqs=2, batch=2)
    out = ctx.response_at_freqs(dev(sc.g, torch.float64), oms, sc.T, rtol=1e-11, method="split2", plane=sc.plane,
                                want_full=True)
    for f, W in enumerate(oms):
        want = exact.y_plain(A, sc.g, W, sc.T)
        assert rel(out["Y"][f].cpu().numpy(), want) < 1e-10
        o = periodic.split2(A, sc.g, W, sc.T, periodic.period_multiple(W, sc.T))
        assert rel(out["Y"][f].cpu().numpy(), o) < 1e-10
        Pw = yee.plane_fields(sc.grid, want, sc.plane)
        assert rel(out["E_plane"][f].cpu().numpy(), Pw) < 1e-10
    ctx.close()


def test_split2_fp32_3d_and_batching():
    sc = S.config_3d(n=16, fill=0.3, T=45.0)
    A = yee.Operator(sc.grid, sc.eps_cell).matrix()
    oms = S.freq_list(3)
    g = dev(sc.g, torch.float32)
    ctx = Context(sc.grid, sc.eps_cell, precision="fp32", krylov_dim=32, max_freqs=3, batch=3)
    out = ctx.response_at_freqs(g, oms, sc.T, rtol=1e-7, method="split2", plane=sc.plane, want_full=True)
    ctx.close()
    for f, W in enumerate(oms):
        assert rel(out["Y"][f].double().cpu().numpy(), exact.y_plain(A, sc.g, W, sc.T)) < 1e-6
    # one frequency at a time gives the same bits as the batch
    ctx1 = Context(sc.grid, sc.eps_cell, precision="fp32", krylov_dim=32, max_freqs=1, batch=1)
    one = ctx1.response_at_freqs(g, oms[1:2], sc.T, rtol=1e-7, method="split2", plane=sc.plane, want_full=True)
    ctx1.close()
    assert torch.equal(one["Y"][0], out["Y"][1])


@pytest.mark.parametrize("batch", [4, 2])
def test_split4d_matches_oracle_and_saves_matvecs(batch):
    """Close neighbouring frequencies (step 0.001, as in the paper's
    experiments): every response equals the exact one, and the transients
    of the differences need fewer Krylov steps than the transients of Im z
    themselves.  batch 2 hands the last transient of a wave to the next."""
    sc = S.config_2d(n=12, ndisks=2, T=60.0)
    A = yee.Operator(sc.grid, sc.eps_cell).matrix()
    W0 = 2 * np.pi / 16
    oms = [W0, W0 * 1.001, W0 * 1.002, W0 * 1.003]
    g = dev(sc.g, torch.float64)
    ctx = Context(sc.grid, sc.eps_cell, precision="fp64", krylov_dim=40, max_freqs=4, batch=batch)
    ctx.reset_stats()
    a = ctx.response_at_freqs(g, oms, sc.T, rtol=1e-11, method="split4d", plane=sc.plane, want_full=True)
    st4 = ctx.stats()
    ctx.reset_stats()
    b = ctx.response_at_freqs(g, oms, sc.T, rtol=1e-11, method="split", plane=sc.plane, want_full=True)
    st1 = ctx.stats()
    ctx.close()
    ys, _, _ = periodic.split1_next(A, sc.g, oms, sc.T)
    for f, W in enumerate(oms):
        want = exact.y_plain(A, sc.g, W, sc.T)
        assert rel(a["Y"][f].cpu().numpy(), want) < 1e-10
        assert rel(a["Y"][f].cpu().numpy(), ys[f]) < 1e-10
        assert rel(a["Y"][f].cpu().numpy(), b["Y"][f].cpu().numpy()) < 1e-10
    assert st4["substeps"] < st1["substeps"]
