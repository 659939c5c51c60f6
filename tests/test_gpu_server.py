"""The request server: continuous batching of 1D and 2D solves over one device arena.

Each request's result must be the same bits alone and in any mix (its arithmetic depends
only on its own data and its own time step), equal to the batch solve of the same
instance, and the server must admit requests only as arena space frees up."""
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


def _drain(srv, max_steps=16, limit=100000):
    res = []
    for _ in range(limit):
        act, q = srv.step(max_steps)
        res += srv.poll()
        if act == 0 and q == 0:
            break
    return res


@pytest.mark.parametrize("precision", [0, 1])
def test_alone_equals_mixed_and_batch(npw, precision):
    p = npw.Params(rbf=npw.NPW_RBF_GA, precision=precision, batch_mode=1)
    target = I.burgers_batch(count=1, nmin=2500, nmax=2600, seed_index=7)[0]
    others = I.burgers_batch(count=8, nmin=64, nmax=5000, seed_index=8)
    # alone
    srv = npw.Server(heap_cells=200000, max_slots=16, params=p)
    srv.submit(target.u0[0], npw.NPW_FLUX_BURGERS, 0, target.dx, 0.4, 0.5, tag=1)
    alone = _drain(srv)[0]
    srv.close()
    # in a mix: others start first, the target arrives while they run, more arrive later
    srv = npw.Server(heap_cells=200000, max_slots=16, params=p)
    for it in others[:5]:
        srv.submit(it.u0[0], npw.NPW_FLUX_BURGERS, 0, it.dx, 0.3, 0.5, tag=0)
    got = []
    for _ in range(3):
        srv.step(8)
        got += srv.poll()
    srv.submit(target.u0[0], npw.NPW_FLUX_BURGERS, 0, target.dx, 0.4, 0.5, tag=1)
    srv.step(5)
    got += srv.poll()
    for it in others[5:]:
        srv.submit(it.u0[0], npw.NPW_FLUX_BURGERS, 0, it.dx, 0.2, 0.5, tag=0)
    got += _drain(srv, max_steps=7)
    mixed = [r for r in got if r["tag"] == 1][0]
    assert alone["status"] == 0 and mixed["status"] == 0
    assert alone["steps"] == mixed["steps"]
    assert np.array_equal(alone["u"], mixed["u"])
    # the same instance through the batch solve
    table, _ = npw.make_instances([target.n], [target.dx], [0.4], [0.5], [0])
    dt = torch.float32 if precision == 1 else torch.float64
    arena = torch.tensor(target.u0[0], dtype=dt, device="cuda")
    st, stats = npw.npweno_batch_solve(arena, table, 1, npw.NPW_FLUX_BURGERS, p)
    assert st == 0 and stats[0]["steps"] == alone["steps"]
    assert np.array_equal(arena.cpu().numpy(), alone["u"])
    assert len([r for r in got if r["status"] == 0]) == 9


def test_fp64_server_matches_oracle(npw):
    p = npw.Params(precision=0)
    srv = npw.Server(heap_cells=50000, max_slots=8, params=p)
    insts = I.burgers_batch(count=4, nmin=100, nmax=900, seed_index=9)
    for k, it in enumerate(insts):
        srv.submit(it.u0[0], npw.NPW_FLUX_BURGERS, 0, it.dx, 0.2, 0.5, tag=k)
    res = sorted(_drain(srv), key=lambda r: r["tag"])
    for it, r in zip(insts, res):
        ref, rst = O.solve(it.u0[0], it.dx, 0.2, 0.5, O.BURGERS, O.PERIODIC, O.Params())
        assert r["steps"] == rst["steps"]
        assert np.abs(r["u"] - ref).max() <= 1e-11 * np.abs(ref).max()


def test_admission_by_memory_and_mixed_kinds(npw):
    """The heap holds about two requests at a time; eight (Burgers and Euler) all finish, each
    identical to its own batch solve."""
    p = npw.Params(rbf=npw.NPW_RBF_MQ, precision=1, batch_mode=1)
    burg = I.burgers_batch(count=4, nmin=1900, nmax=2000, seed_index=10)
    eul = I.euler_batch(count=4, nmin=600, nmax=650, seed_index=11)
    srv = npw.Server(heap_cells=4100, max_slots=8, params=p)
    for k, it in enumerate(burg):
        srv.submit(it.u0[0], npw.NPW_FLUX_BURGERS, 0, it.dx, 0.1, 0.5, tag=k)
    for k, it in enumerate(eul):
        srv.submit(it.u0.ravel(), npw.NPW_FLUX_EULER1D, 1, it.dx, min(it.t_end, 0.02), 0.5, tag=10 + k)
    got, max_active = [], 0
    for _ in range(100000):
        act, q = srv.step(6)
        max_active = max(max_active, act)
        got += srv.poll()
        if act == 0 and q == 0:
            break
    assert len(got) == 8 and all(r["status"] == 0 for r in got)
    assert max_active <= 2
    for r in got:
        if r["tag"] < 10:
            it, m, kind, bc, te = burg[r["tag"]], 1, npw.NPW_FLUX_BURGERS, 0, 0.1
        else:
            it, m, kind, bc, te = eul[r["tag"] - 10], 3, npw.NPW_FLUX_EULER1D, 1, min(eul[r["tag"] - 10].t_end, 0.02)
        table, _ = npw.make_instances([it.n], [it.dx], [te], [0.5], [bc], m=m)
        arena = torch.tensor(it.u0.ravel(), dtype=torch.float32, device="cuda")
        st, stats = npw.npweno_batch_solve(arena, table, m, kind, p)
        assert np.array_equal(arena.cpu().numpy(), r["u"])


def test_failed_request_does_not_disturb_others(npw):
    p = npw.Params(precision=1, batch_mode=1)
    srv = npw.Server(heap_cells=20000, max_slots=4, params=p)
    good = I.burgers_batch(count=2, nmin=500, nmax=900, seed_index=12)
    bad = good[0].u0[0].copy()
    bad[10] = np.nan
    srv.submit(good[0].u0[0], npw.NPW_FLUX_BURGERS, 0, good[0].dx, 0.2, 0.5, tag=0)
    srv.submit(bad, npw.NPW_FLUX_BURGERS, 0, good[0].dx, 0.2, 0.5, tag=1)
    srv.submit(good[1].u0[0], npw.NPW_FLUX_BURGERS, 0, good[1].dx, 0.2, 0.5, tag=2)
    res = {r["tag"]: r for r in _drain(srv)}
    assert res[1]["status"] == npw.NPW_ENONFINITE
    assert res[0]["status"] == 0 and res[2]["status"] == 0 and res[2]["t"] == 0.2
    with pytest.raises(npw.NpwError) as e:
        srv.submit(np.ones(5), npw.NPW_FLUX_BURGERS, 0, 0.1, 0.2, 0.5)
    assert e.value.status == npw.NPW_EINVAL
    for _ in range(4):
        srv.submit(good[0].u0[0], npw.NPW_FLUX_BURGERS, 0, good[0].dx, 0.2, 0.5)
    with pytest.raises(npw.NpwError) as e:
        srv.submit(good[0].u0[0], npw.NPW_FLUX_BURGERS, 0, good[0].dx, 0.2, 0.5)
    assert e.value.status == npw.NPW_EBUSY
    _drain(srv)


@pytest.mark.parametrize("precision", [0, 1])
def test_2d_requests_alone_equal_the_2d_solve(npw, precision):
    """2D requests (Euler vortex and four-quadrant data, k = 3; the Sec. 7 Example 2 advection
    with a per-direction boundary, k = 2 on the cross) served between 1D requests: each result
    equals npweno_solve_2d of the same domain bit for bit, with the same step count."""
    p = npw.Params(rbf=npw.NPW_RBF_GA, precision=precision, batch_mode=1)
    dtype = torch.float32 if precision else torch.float64
    doms = I.euler2d_batch(40, 2, seed_index=11)
    n2 = 36
    edges = np.linspace(0, 1, n2 + 1)
    ex2 = np.repeat(np.where(edges[1:] <= 0.5, 1.0, -1.0)[:, None], n2, axis=1)[None]
    reqs = [(doms[0][0], npw.NPW_FLUX_EULER2D, npw.NPW_BC_PERIODIC, -1, doms[0][1], 0.3, p),
            (doms[1][0], npw.NPW_FLUX_EULER2D, npw.NPW_BC_TRANSMISSIVE, -1, doms[1][1], 0.05, p)]
    pk2 = npw.Params(k=2, scheme=npw.NPW_RBF_ENO, cross_2d=1, precision=precision, inflow=(1.0, 0, 0, 0), batch_mode=1)
    # standalone references
    refs = []
    for U, kind, bc, bcy, d, t, pp in reqs:
        u = torch.tensor(U, dtype=dtype, device="cuda")
        st = npw.npweno_solve_2d(u, d, d, t, 0.4, kind, bc, pp)
        refs.append((u.cpu().numpy(), st))
    u = torch.tensor(ex2, dtype=dtype, device="cuda")
    pk2_ref = npw.Params(**{**pk2.__dict__, "bc_y": npw.NPW_BC_INFLOW})
    st = npw.npweno_solve_2d(u, 1.0 / n2, 1.0 / n2, 0.2, 0.4, npw.NPW_FLUX_ADVECTION, npw.NPW_BC_PERIODIC, pk2_ref)
    ref_ex2 = (u.cpu().numpy(), st)
    torch.cuda.synchronize()
    # served in a mix with 1D requests (the server's method parameters are those of the Euler
    # requests; the Example 2 request goes to its own k = 2 server)
    ones = I.burgers_batch(count=4, nmin=64, nmax=3000, seed_index=12)
    srv = npw.Server(heap_cells=60000, max_slots=8, params=p)
    srv.submit(ones[0].u0[0], npw.NPW_FLUX_BURGERS, 0, ones[0].dx, 0.3, 0.5, tag=100)
    srv.step(4)
    got = srv.poll()
    for i, (U, kind, bc, bcy, d, t, _) in enumerate(reqs):
        srv.submit(U, kind, bc, d, t, 0.4, tag=i + 1, dy=d, bc_y=bcy)
        srv.submit(ones[i + 1].u0[0], npw.NPW_FLUX_BURGERS, 0, ones[i + 1].dx, 0.2, 0.5, tag=200 + i)
        srv.step(3)
        got += srv.poll()
    got += _drain(srv, max_steps=5)
    srv.close()
    by_tag = {r["tag"]: r for r in got}
    assert all(r["status"] == 0 for r in got) and len(by_tag) == 5
    for i, (ref, st) in enumerate(refs):
        r = by_tag[i + 1]
        assert r["steps"] == st["steps"]
        assert np.array_equal(r["u"], ref.astype(r["u"].dtype))
    srv = npw.Server(heap_cells=20000, max_slots=4, params=pk2)
    srv.submit(ones[3].u0[0], npw.NPW_FLUX_BURGERS, 0, ones[3].dx, 0.1, 0.5, tag=300)
    srv.submit(ex2, npw.NPW_FLUX_ADVECTION, npw.NPW_BC_PERIODIC, 1.0 / n2, 0.2, 0.4, tag=9, dy=1.0 / n2,
               bc_y=npw.NPW_BC_INFLOW)
    res = {r["tag"]: r for r in _drain(srv, max_steps=6)}
    srv.close()
    assert res[9]["status"] == 0 and res[9]["steps"] == ref_ex2[1]["steps"]
    assert np.array_equal(res[9]["u"], ref_ex2[0].astype(res[9]["u"].dtype))


def test_2d_request_validation(npw):
    p = npw.Params(batch_mode=1)
    srv = npw.Server(heap_cells=5000, max_slots=2, params=p)
    u = np.zeros((4, 8, 8))
    with pytest.raises(npw.NpwError):  # 1D Euler flux in 2D
        srv.submit(u, npw.NPW_FLUX_EULER1D, 0, 0.1, 0.1, 0.4, dy=0.1)
    with pytest.raises(npw.NpwError):  # 2D Euler flux in 1D
        srv.submit(u, npw.NPW_FLUX_EULER2D, 0, 0.1, 0.1, 0.4)
    with pytest.raises(npw.NpwError):  # larger than the heap
        srv.submit(np.zeros((4, 40, 40)), npw.NPW_FLUX_EULER2D, 0, 0.1, 0.1, 0.4, dy=0.1)
    with pytest.raises(npw.NpwError):  # bad y boundary
        srv.submit(u, npw.NPW_FLUX_EULER2D, 0, 0.1, 0.1, 0.4, dy=0.1, bc_y=9)
    srv.close()


def test_per_request_precision_lanes(npw):
    """One server, requests of both tolerance classes interleaved: the loose ones run in the
    mixed lane, the strict ones in the FP64 lane, each equal bit for bit to the solve of the same
    request in its precision (npweno_batch_solve with the per-stage kernels, npweno_solve_2d), and
    the FP64 ones match the oracle."""
    p = npw.Params(rbf=npw.NPW_RBF_GA, precision=npw.NPW_FP32_MIXED, batch_mode=1)
    burg = I.burgers_batch(count=6, nmin=100, nmax=3000, seed_index=13)
    U, d = I.euler2d_batch(40, 1, seed_index=14)[0]
    srv = npw.Server(heap_cells=40000, max_slots=12, params=p)
    tols = [1e-3, 1e-10, 0.0, 1e-8, 5e-4, 1e-12]
    for k, (it, tol) in enumerate(zip(burg, tols)):
        srv.submit(it.u0[0], npw.NPW_FLUX_BURGERS, 0, it.dx, 0.3, 0.5, tag=k, tolerance=tol)
        srv.step(3)
    srv.submit(U, npw.NPW_FLUX_EULER2D, 0, d, 0.2, 0.4, tag=50, dy=d, tolerance=1e-10)
    srv.submit(U, npw.NPW_FLUX_EULER2D, 0, d, 0.2, 0.4, tag=51, dy=d, tolerance=1e-3)
    res = {r["tag"]: r for r in srv.poll() + _drain(srv, max_steps=5)}
    srv.close()
    assert len(res) == 8 and all(r["status"] == 0 for r in res.values())
    for k, (it, tol) in enumerate(zip(burg, tols)):
        r = res[k]
        prec = npw.NPW_FP32_MIXED if (tol == 0.0 or tol >= 1e-4) else npw.NPW_FP64
        assert r["precision"] == prec
        pk = npw.Params(rbf=npw.NPW_RBF_GA, precision=prec, batch_mode=1)
        table, _ = npw.make_instances([it.n], [it.dx], [0.3], [0.5], [0])
        dt = torch.float32 if prec == npw.NPW_FP32_MIXED else torch.float64
        arena = torch.tensor(it.u0[0], dtype=dt, device="cuda")
        st, stats = npw.npweno_batch_solve(arena, table, 1, npw.NPW_FLUX_BURGERS, pk)
        assert st == 0 and stats[0]["steps"] == r["steps"]
        assert np.array_equal(arena.cpu().numpy(), r["u"])
        if prec == npw.NPW_FP64:
            ref, rst = O.solve(it.u0[0], it.dx, 0.3, 0.5, O.BURGERS, O.PERIODIC, O.Params(rbf=O.GA))
            assert rst["steps"] == r["steps"] and np.abs(r["u"] - ref).max() <= 1e-11 * np.abs(ref).max()
    for tag, prec in ((50, npw.NPW_FP64), (51, npw.NPW_FP32_MIXED)):
        r = res[tag]
        assert r["precision"] == prec
        dt = torch.float32 if prec == npw.NPW_FP32_MIXED else torch.float64
        u = torch.tensor(U, dtype=dt, device="cuda")
        st = npw.npweno_solve_2d(u, d, d, 0.2, 0.4, npw.NPW_FLUX_EULER2D, 0,
                                 npw.Params(rbf=npw.NPW_RBF_GA, precision=prec))
        assert st["steps"] == r["steps"] and np.array_equal(u.cpu().numpy(), r["u"])


def test_lanes_run_independently(npw):
    """Each precision lane runs its rounds on its own stream: a float request admitted while the
    FP64 lane works through long rounds (a 512^2 2D Euler square, 16 steps a round) comes back
    in well under one FP64 round (its launches run between the FP64 lane's, at the greater
    stream priority), while the FP64 request is still running; both results equal their solves
    alone."""
    p = npw.Params(rbf=npw.NPW_RBF_GA, precision=npw.NPW_FP32_MIXED, batch_mode=1)
    U, d = I.euler2d_batch(512, 1, seed_index=15)[0]
    small = I.burgers_batch(count=1, nmin=128, nmax=130, seed_index=16)[0]
    srv = npw.Server(heap_cells=2_000_000, max_slots=8, params=p)
    t64 = 200 * 0.05 * d
    srv.submit(U, npw.NPW_FLUX_EULER2D, 0, d, t64, 0.4, tag=64, dy=d, tolerance=1e-10)
    got = []
    for _ in range(3):  # the FP64 lane is in its rounds
        srv.step(16)
        got += srv.poll()
    srv.submit(small.u0[0], npw.NPW_FLUX_BURGERS, 0, small.dx, 0.01, 0.5, tag=32, tolerance=1e-3)
    for _ in range(100000):
        srv.step(16)
        got += srv.poll()
        if any(r["tag"] == 32 for r in got):
            break
    assert [r["tag"] for r in got] == [32], got  # the FP64 request is still running
    got += _drain(srv, max_steps=16)
    srv.close()
    by_tag = {r["tag"]: r for r in got}
    r64, r32 = by_tag[64], by_tag[32]
    assert r64["status"] == 0 and r64["precision"] == npw.NPW_FP64 and r32["precision"] == npw.NPW_FP32_MIXED
    t_round64 = (r64["done_s"] - r64["admit_s"]) / -(-r64["steps"] // 16)
    lat32 = r32["done_s"] - r32["submit_s"]
    assert lat32 < 0.6 * t_round64, (lat32, t_round64, r64["steps"])
    u = torch.tensor(U, dtype=torch.float64, device="cuda")
    st = npw.npweno_solve_2d(u, d, d, t64, 0.4, npw.NPW_FLUX_EULER2D, 0,
                             npw.Params(rbf=npw.NPW_RBF_GA, precision=npw.NPW_FP64))
    assert st["steps"] == r64["steps"] and np.array_equal(u.cpu().numpy(), r64["u"])
    table, _ = npw.make_instances([small.n], [small.dx], [0.01], [0.5], [0])
    arena = torch.tensor(small.u0[0], dtype=torch.float32, device="cuda")
    st, stats = npw.npweno_batch_solve(arena, table, 1, npw.NPW_FLUX_BURGERS, p)
    assert stats[0]["steps"] == r32["steps"] and np.array_equal(arena.cpu().numpy(), r32["u"])
