"""GPU parity of the batched restart in Krylov dimension (kx_batch_create,
response_restart_dim_batch): one launch per Arnoldi phase for every problem
of an uneven batch (Sect. 3.4, Fig. alg:rst on each problem).

Each problem's output-plane intensities are compared with the same problem
solved alone by response_restart_dim (same method; the batched launches
split the blocks differently, so FP32 reductions run in another order) and
with the oracle's exact response (the FP32 response target, 1e-6 on the
fields, is 2e-6 on their squared sum).
"""
import numpy as np
import pytest

import scenario as S
from oracle import exact, yee

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

from paper_1707_00023_gb300 import Batch, Context, KxError  # noqa: E402
from paper_1707_00023_gb300._binding import KX_EINVAL  # noqa: E402

T, M, NF = 15.0, 24, 2


def contexts(scs, **kw):
    return [Context(sc.grid, sc.eps_cell, precision="fp32", krylov_dim=M, max_freqs=NF, batch=2, stream="own",
                    rst_samples=4000, **kw) for sc in scs]


def test_batch_matches_single_problems_and_oracle():
    scs = S.config_uneven(count=4, seed=6, nmin=8, nmax=20, T=T, m=M, nfreq=NF, step=4)
    assert all(sc.grid.n[0] % 4 == 0 for sc in scs) and len({sc.grid.n for sc in scs}) > 1
    ctxs = contexts(scs)
    gs = [torch.tensor(sc.g, dtype=torch.float32, device="cuda") for sc in scs]
    oms = np.stack([sc.omegas for sc in scs])
    planes = np.array([sc.plane for sc in scs])
    b = Batch(ctxs)
    info = b.info()
    assert info["problems"] == 4 and info["sweep_tiles_per_block"] in (1, 2, 4, 8, 16)
    inten, resid, rst = b.response(gs, oms, T, rtol=1e-7, planes=planes)
    assert np.all(resid <= 1e-7) and np.all(rst >= 1)
    first = b.info()
    assert first["batched_launches"] > 0
    # each restart's batched process ran as a replay of its captured graph
    assert first["graph_replays"] >= int(rst.max())
    for i, sc in enumerate(scs):
        alone = ctxs[i].response_restart_dim(gs[i], sc.omegas, T, rtol=1e-7, plane=sc.plane)
        # the stopping test may fall one restart apart under another reduction order
        assert np.all(np.abs(alone["restarts"] - rst[i]) <= 1)
        A = yee.Operator(sc.grid, sc.eps_cell).matrix()
        for f in range(NF):
            assert abs(inten[i, f] - alone["intensity"][f]) < 2e-6 * alone["intensity"][f]
            want = yee.intensity(sc.grid, exact.y_plain(A, sc.g, sc.omegas[f], T), sc.plane)
            assert abs(inten[i, f] - want) < 2e-6 * want
    # the same call again gives the same bits (fixed block split and reduction order),
    # also with the batched sweep launches timed by events (launched directly, not
    # as graph replays)
    b.set_timing(True)
    again, _, _ = b.response(gs, oms, T, rtol=1e-7, planes=planes)
    b.set_timing(False)
    np.testing.assert_array_equal(again, inten)
    ti = b.info()
    assert ti["sweep_timed_launches"] > 0 and ti["sweep_ms"] > 0.0 and ti["sweep_bytes"] > 0.0
    assert ti["graph_replays"] == first["graph_replays"]
    b.close()
    # a second batch of the same size class takes the tuned split from the cache
    b2 = Batch(ctxs)
    assert b2.info()["from_cache"] == 1
    assert b2.info()["sweep_tiles_per_block"] == info["sweep_tiles_per_block"]
    b2.close()
    for c in ctxs:
        c.close()


def test_batch_zero_source_member_and_refusals():
    scs = S.config_uneven(count=3, seed=9, nmin=8, nmax=16, T=T, m=M, nfreq=NF, step=4)
    ctxs = contexts(scs)
    gs = [torch.tensor(sc.g, dtype=torch.float32, device="cuda") for sc in scs]
    gs[1] = torch.zeros_like(gs[1])
    oms = np.stack([sc.omegas for sc in scs])
    planes = np.array([sc.plane for sc in scs])
    b = Batch(ctxs)
    inten, _, rst = b.response(gs, oms, T, rtol=1e-7, planes=planes)
    assert np.all(inten[1] == 0.0) and np.all(rst[1] == 0)
    for i in (0, 2):
        alone = ctxs[i].response_restart_dim(gs[i], scs[i].omegas, T, rtol=1e-7, plane=scs[i].plane)
        assert np.all(np.abs(inten[i] - alone["intensity"]) < 2e-6 * alone["intensity"])
    b.close()
    # contexts that do not qualify are refused with a reason
    grid = S.Grid(3, (10, 8, 8), (S.PERIODIC, S.PERIODIC, S.PEC), 2, 2, 1.0)
    odd = Context(grid, np.ones(grid.shape), precision="fp32", krylov_dim=M, max_freqs=NF, batch=2,
                  rst_samples=4000)
    with pytest.raises(KxError, match="multiple of 4") as e:
        Batch([ctxs[0], odd])
    assert e.value.status == KX_EINVAL
    with pytest.raises(KxError, match="twice"):
        Batch([ctxs[0], ctxs[0]])
    one_slot = Context(scs[0].grid, scs[0].eps_cell, precision="fp32", krylov_dim=M, max_freqs=NF, batch=1,
                       rst_samples=4000)
    with pytest.raises(KxError, match="batch >= 2"):
        Batch([one_slot])
    for c in ctxs + [odd, one_slot]:
        c.close()
