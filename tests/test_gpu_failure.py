"""Failure paths of the solve loops, made without a GPU fault.

* Device side: every solve has a step limit (npw_params.max_steps, or the automatic one); a run
  that reaches it ends with NPW_ETIMEOUT in its own status word, with the steps it took, instead
  of looping on the device.  Covered for the resident whole-solve kernel, the per-stage kernels
  (FP64 and mixed), a batch where only one instance runs out, the 2D solve and the server.
* Host side: every wait of the library on its stream is bounded (NPW_WAIT_TIMEOUT_S, seconds).
  A limit shorter than the solve makes the call return NPW_ETIMEOUT while its launches are still
  queued; the device stays usable: after a plain synchronisation the next solve matches the
  oracle.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1602_00182_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def npw():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1602_00182_gb300 import build as b
    b.build()
    import paper_1602_00182_gb300.npweno as m
    m.load()
    return m


@pytest.mark.parametrize("precision,batch_mode", [(0, 0), (1, 0), (1, 1)])
def test_step_limit_ends_a_solve(npw, precision, batch_mode):
    """Burgers instances that need hundreds of steps, with max_steps = 7: the batch returns
    NPW_ETIMEOUT, each instance stops after exactly 7 steps short of t_end; without the limit
    the same batch finishes (mixed, batch_mode 0: the resident kernel)."""
    inst = I.burgers_batch(count=3, nmin=500, nmax=3000, seed_index=9)
    ns = [it.n for it in inst]
    table, total = npw.make_instances(ns, [it.dx for it in inst], [1.0] * 3, [0.5] * 3, [0] * 3)
    dtype = torch.float64 if precision == 0 else torch.float32
    host = np.concatenate([it.u0[0] for it in inst])
    arena = torch.tensor(host, dtype=dtype, device="cuda")
    p = npw.Params(rbf=npw.NPW_RBF_GA, precision=precision, batch_mode=batch_mode, max_steps=7)
    st, stats = npw.npweno_batch_solve(arena, table, 1, npw.NPW_FLUX_BURGERS, p, raise_on_error=False)
    assert st == npw.NPW_ETIMEOUT
    for s in stats:
        assert s["status"] == npw.NPW_ETIMEOUT and s["steps"] == 7 and 0.0 < s["t"] < 1.0
    assert torch.isfinite(arena).all()
    arena = torch.tensor(host, dtype=dtype, device="cuda")
    p.max_steps = 0
    st, stats = npw.npweno_batch_solve(arena, table, 1, npw.NPW_FLUX_BURGERS, p)
    assert st == 0 and all(s["t"] == 1.0 and s["steps"] > 7 for s in stats)


def test_step_limit_stops_only_the_instance_that_reaches_it(npw):
    """Each instance has its own step count: with max_steps = 40 the instance that needs more
    steps runs out, the short ones finish normally."""
    ns = [64, 128, 2048]
    dxs = [2 * np.pi / n for n in ns]
    table, total = npw.make_instances(ns, dxs, [0.05, 0.05, 1.0], [0.5] * 3, [0] * 3)
    host = np.concatenate([1.0 + 0.5 * np.sin(2 * np.pi * np.arange(n) / n) for n in ns])
    arena = torch.tensor(host, dtype=torch.float64, device="cuda")
    st, stats = npw.npweno_batch_solve(arena, table, 1, npw.NPW_FLUX_BURGERS, npw.Params(max_steps=40),
                                       raise_on_error=False)
    assert st == npw.NPW_ETIMEOUT
    assert stats[0]["status"] == 0 and stats[0]["t"] == 0.05
    assert stats[1]["status"] == 0 and stats[1]["t"] == 0.05
    assert stats[2]["status"] == npw.NPW_ETIMEOUT and stats[2]["steps"] == 40


def test_step_limit_2d(npw):
    U, d = I.isentropic_vortex(48, 4.0, 5.0, 5.0)
    u = torch.tensor(U, dtype=torch.float64, device="cuda")
    with pytest.raises(npw.NpwError) as e:
        npw.npweno_solve_2d(u, d, d, 5.0, 0.5, npw.NPW_FLUX_EULER2D, 0, npw.Params(max_steps=3))
    assert e.value.status == npw.NPW_ETIMEOUT
    assert torch.isfinite(u).all()


def test_host_wait_limit_returns_and_device_stays_usable(npw, monkeypatch):
    """NPW_WAIT_TIMEOUT_S = 1 ms around a solve of ~1 s: the call returns NPW_ETIMEOUT with its
    launches still queued; a plain synchronisation lets them finish, and the next solve (default
    limit) matches the oracle bit for bit."""
    inst = I.burgers_batch(count=1, nmin=6000, nmax=6001, seed_index=2)[0]
    u = torch.tensor(inst.u0[0], dtype=torch.float64, device="cuda")
    monkeypatch.setenv("NPW_WAIT_TIMEOUT_S", "0.001")
    with pytest.raises(npw.NpwError) as e:
        npw.npweno_solve(u, inst.dx, 1.5, 0.5, npw.NPW_FLUX_BURGERS, 0, npw.Params(rbf=npw.NPW_RBF_GA))
    assert e.value.status == npw.NPW_ETIMEOUT
    torch.cuda.synchronize()
    monkeypatch.delenv("NPW_WAIT_TIMEOUT_S")
    u0, dx = I.advection_sin(101)
    g = torch.tensor(u0, dtype=torch.float64, device="cuda")
    st = npw.npweno_solve(g, dx, 0.4, 0.5, npw.NPW_FLUX_ADVECTION, 0, npw.Params())
    ref, rst = O.solve(u0, dx, 0.4, 0.5, O.ADVECTION, O.PERIODIC, O.Params())
    assert st["steps"] == rst["steps"]
    assert np.abs(g.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
