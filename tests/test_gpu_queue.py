"""The work-queue batch (npweno_queue_solve): uneven 1D and 2D instances of several flux kinds in
one persistent kernel per stage.

Each item runs the same per-item body as the one-CTA-per-item kernels, and an instance's
arithmetic depends only on its own data, so every instance must come out bit for bit as when
it is solved on its own (npweno_batch_solve for 1D, npweno_solve_2d for 2D), whatever else
shares the queue; the FP64 queue must also match the oracle (1e-11 relative on these runs).
"""
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


def _mix(npw, small=False):
    """A mix of periodic Burgers, transmissive 1D Euler, 2D Euler (vortex, four-quadrant) and 2D
    advection instances of uneven sizes, with their initial fields."""
    specs, fields = [], []
    for it in I.burgers_batch(count=4, nmin=64, nmax=900 if small else 6000, seed_index=41):
        specs.append(dict(kind=npw.NPW_FLUX_BURGERS, nx=it.n, dx=it.dx, t_end=0.3, cfl=0.5, bc=0))
        fields.append(it.u0.ravel())
    for it in I.euler_batch(count=2, nmin=300, nmax=700 if small else 9000, seed_index=42):
        specs.append(dict(kind=npw.NPW_FLUX_EULER1D, nx=it.n, dx=it.dx, t_end=min(it.t_end, 0.03), cfl=0.5, bc=1))
        fields.append(it.u0.ravel())
    for n2 in ((40, 37) if small else (96, 200)):
        for U, d in I.euler2d_batch(n2, 2, seed_index=43):
            specs.append(dict(kind=npw.NPW_FLUX_EULER2D, nx=n2, ny=n2, dx=d, dy=d, t_end=0.02 if d < 0.05 else 0.2,
                              cfl=0.5, bc=0))
            fields.append(U.ravel())
    nx, ny = (30, 22) if small else (150, 70)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    A = 1.0 + 0.5 * np.sin(2 * np.pi * x)[None, :] * np.cos(2 * np.pi * y)[:, None]
    specs.append(dict(kind=npw.NPW_FLUX_ADVECTION, nx=nx, ny=ny, dx=1.0 / nx, dy=1.0 / ny, t_end=0.1, cfl=0.4, bc=0))
    fields.append(A.ravel())
    return specs, fields


def _alone(npw, sp, u0, p, dtype):
    """The instance solved on its own through its own entry point."""
    if sp.get("ny", 0):
        m = 4 if sp["kind"] == npw.NPW_FLUX_EULER2D else 1
        u = torch.tensor(u0.reshape(m, sp["ny"], sp["nx"]), dtype=dtype, device="cuda")
        st = npw.npweno_solve_2d(u, sp["dx"], sp["dy"], sp["t_end"], sp["cfl"], sp["kind"], sp["bc"], p)
        return u.cpu().numpy().ravel(), st
    m = 3 if sp["kind"] == npw.NPW_FLUX_EULER1D else 1
    table, _ = npw.make_instances([sp["nx"]], [sp["dx"]], [sp["t_end"]], [sp["cfl"]], [sp["bc"]], m=m)
    u = torch.tensor(u0, dtype=dtype, device="cuda")
    st, stats = npw.npweno_batch_solve(u, table, m, sp["kind"], p)
    assert st == 0
    return u.cpu().numpy().ravel(), stats[0]


@pytest.mark.parametrize("precision,batch_mode", [(1, 0), (1, 1), (0, 0)])
def test_queue_mix_equals_each_instance_alone(npw, precision, batch_mode):
    """FP64 runs drop faces with |eta| > 100: with the printed eta the 200^2 four-quadrant
    instance becomes non-finite in FP64 (the oracle's own run too), from a single face whose
    Table k3 denominator vanishes; the bound drops that face only."""
    specs, fields = _mix(npw)
    table, total, offs = npw.make_queue_instances(specs)
    dtype = torch.float64 if precision == 0 else torch.float32
    arena = torch.tensor(np.concatenate(fields), dtype=dtype, device="cuda")
    p = npw.Params(rbf=npw.NPW_RBF_GA, precision=precision, batch_mode=batch_mode,
                   eta_max=100.0 if precision == 0 else 0.0)
    st, stats = npw.npweno_queue_solve(arena, table, p)
    assert st == 0
    a = arena.cpu().numpy()
    for sp, u0, off, s in zip(specs, fields, offs, stats):
        ref, rs = _alone(npw, sp, u0, p, dtype)
        got = a[off:off + ref.size]
        assert s["status"] == 0 and s["t"] == sp["t_end"]
        assert s["steps"] == rs["steps"] and s["alpha_max"] == rs["alpha_max"], (sp["kind"], sp["nx"])
        assert np.array_equal(got, ref), (sp["kind"], sp["nx"], np.abs(got - ref).max())
        assert s["eta"] == rs["eta"]


def test_queue_fp64_matches_oracle(npw):
    specs, fields = _mix(npw, small=True)
    table, total, offs = npw.make_queue_instances(specs)
    arena = torch.tensor(np.concatenate(fields), dtype=torch.float64, device="cuda")
    op = O.Params(rbf=O.GA)
    p = npw.Params(rbf=npw.NPW_RBF_GA)
    st, stats = npw.npweno_queue_solve(arena, table, p)
    assert st == 0
    a = arena.cpu().numpy()
    for sp, u0, off, s in zip(specs, fields, offs, stats):
        if sp.get("ny", 0):
            m = 4 if sp["kind"] == npw.NPW_FLUX_EULER2D else 1
            ref, rs = O.solve_2d(u0.reshape(m, sp["ny"], sp["nx"]), sp["dx"], sp["dy"], sp["t_end"], sp["cfl"],
                                 sp["kind"], sp["bc"], op)
        else:
            m = 3 if sp["kind"] == npw.NPW_FLUX_EULER1D else 1
            ref, rs = O.solve(u0.reshape(m, sp["nx"]), sp["dx"], sp["t_end"], sp["cfl"], sp["kind"], sp["bc"], op)
        ref = ref.ravel()
        got = a[off:off + ref.size]
        assert s["steps"] == rs["steps"]
        assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max(), (sp["kind"], sp["nx"])
        assert s["eta"] == rs["eta"]


def test_queue_characteristic_euler(npw):
    """Characteristic-wise 1D Euler through the queue equals npweno_batch_solve (face-based
    characteristic body, float state)."""
    inst = I.euler_batch(count=3, nmin=300, nmax=4000, seed_index=44)
    specs = [dict(kind=npw.NPW_FLUX_EULER1D, nx=it.n, dx=it.dx, t_end=min(it.t_end, 0.02), cfl=0.5, bc=1) for it in inst]
    table, total, offs = npw.make_queue_instances(specs)
    fields = [it.u0.ravel() for it in inst]
    arena = torch.tensor(np.concatenate(fields), dtype=torch.float32, device="cuda")
    p = npw.Params(precision=npw.NPW_FP32_MIXED, characteristic=1)
    st, stats = npw.npweno_queue_solve(arena, table, p)
    assert st == 0
    a = arena.cpu().numpy()
    for sp, u0, off, s in zip(specs, fields, offs, stats):
        ref, rs = _alone(npw, sp, u0, p, torch.float32)
        assert s["steps"] == rs["steps"] and np.array_equal(a[off:off + ref.size], ref)


def test_queue_rejects_bad_instances(npw):
    p = npw.Params(characteristic=1)
    table, total, _ = npw.make_queue_instances([dict(kind=npw.NPW_FLUX_BURGERS, nx=100, dx=0.01, t_end=0.1, cfl=0.5)])
    arena = torch.zeros(total, dtype=torch.float64, device="cuda")
    with pytest.raises(npw.NpwError):
        npw.npweno_queue_solve(arena, table, p)
    table, total, _ = npw.make_queue_instances([dict(kind=npw.NPW_FLUX_EULER1D, nx=40, ny=40, dx=0.1, dy=0.1,
                                                     t_end=0.1, cfl=0.5)])
    arena = torch.zeros(total, dtype=torch.float64, device="cuda")
    with pytest.raises(npw.NpwError):  # a 1D flux on a 2D instance
        npw.npweno_queue_solve(arena, table, npw.Params())


def test_queue_step_limit(npw):
    specs, fields = _mix(npw, small=True)
    table, total, offs = npw.make_queue_instances(specs)
    arena = torch.tensor(np.concatenate(fields), dtype=torch.float32, device="cuda")
    p = npw.Params(precision=npw.NPW_FP32_MIXED, batch_mode=1, max_steps=3)
    st, stats = npw.npweno_queue_solve(arena, table, p, raise_on_error=False)
    assert st == npw.NPW_ETIMEOUT
    for s in stats:
        assert s["steps"] <= 3 and s["status"] in (0, npw.NPW_ETIMEOUT)
    assert sum(s["status"] == npw.NPW_ETIMEOUT for s in stats) >= len(stats) // 2
    assert torch.isfinite(arena).all()


@pytest.mark.parametrize("kind", ["burgers", "euler", "advection"])
@pytest.mark.parametrize("bc", [0, 1, 2])
@pytest.mark.parametrize("batch_mode", [0, 1])
def test_queue_fused_step_equals_per_stage(npw, kind, bc, batch_mode):
    """A batch of 1D float instances alone takes one fused launch per RK3 step (u^n loaded once
    with a 9-cell halo, three stages in shared memory, the two state buffers alternating): every
    instance equals the per-stage kernels of npweno_batch_solve (batch_mode 1) bit for bit, with
    the same steps and decision counts.  Sizes from 6 cells (a periodic halo wrapping more than
    once) through several tiles with a ragged end; end times giving odd and even step counts;
    batch_mode 0 also runs the small instances in the resident kernel beside the queue."""
    g = np.random.default_rng(7 + bc)
    ns = [6, 7, 40, 513, 1500, 5000, 9001]
    if kind == "euler":
        kk, m = npw.NPW_FLUX_EULER1D, 3
        fields = []
        for n in ns:
            x = (np.arange(n) + 0.5) / n
            rho = 1.0 + 0.2 * np.sin(2 * np.pi * 3 * x + g.uniform(0, 6)) + 0.5 * (x > 0.6)
            u = 0.3 * np.cos(2 * np.pi * x)
            p = 1.0 + 0.5 * (x < 0.3)
            fields.append(np.concatenate([rho, rho * u, p / 0.4 + 0.5 * rho * u * u]))
    else:
        kk, m = (npw.NPW_FLUX_BURGERS, 1) if kind == "burgers" else (npw.NPW_FLUX_ADVECTION, 1)
        fields = []
        for n in ns:
            x = (np.arange(n) + 0.5) / n
            fields.append(1.0 + 0.5 * np.sin(2 * np.pi * x + g.uniform(0, 6)) + 0.4 * (x > 0.55))
    dxs = [1.0 / n for n in ns]
    t_ends = [0.013 + 0.004 * j for j in range(len(ns))]
    specs = [dict(kind=kk, nx=n, dx=d, t_end=t, cfl=0.5, bc=bc) for n, d, t in zip(ns, dxs, t_ends)]
    table, total, offs = npw.make_queue_instances(specs)
    p = npw.Params(precision=npw.NPW_FP32_MIXED, rbf=npw.NPW_RBF_GA, batch_mode=batch_mode,
                   inflow=(1.3, 0.2, 2.6, 0.0) if kind == "euler" else (1.3, 0, 0, 0))
    arena = torch.tensor(np.concatenate(fields), dtype=torch.float32, device="cuda")
    st, stats = npw.npweno_queue_solve(arena, table, p)
    assert st == 0
    a = arena.cpu().numpy()
    pb = npw.Params(precision=npw.NPW_FP32_MIXED, rbf=npw.NPW_RBF_GA, batch_mode=1, inflow=p.inflow)
    parity = set()
    for sp, u0, off, s in zip(specs, fields, offs, stats):
        tb, _ = npw.make_instances([sp["nx"]], [sp["dx"]], [sp["t_end"]], [sp["cfl"]], [sp["bc"]], m=m)
        u = torch.tensor(u0, dtype=torch.float32, device="cuda")
        stb, rs = npw.npweno_batch_solve(u, tb, m, kk, pb)
        assert stb == 0
        rs = rs[0]
        assert s["status"] == 0 and s["steps"] == rs["steps"] and s["t"] == rs["t"], (sp["nx"], s, rs)
        assert np.array_equal(a[off:off + u0.size], u.cpu().numpy()), (sp["nx"], s["steps"])
        assert s["eta"] == rs["eta"], sp["nx"]
        parity.add(s["steps"] % 2)
    assert parity == {0, 1}


def test_queue_fused_step_mixed_kinds_and_step_limit(npw):
    """1D instances of three flux kinds in one queue batch (the kernel that dispatches per
    item, fused steps): each equals its per-stage solve; with a step limit every instance stops
    after that many fused steps with NPW_ETIMEOUT and its state is the per-stage state after
    the same steps."""
    g = np.random.default_rng(11)
    specs, fields, ms = [], [], []
    for kind, m, n in ((npw.NPW_FLUX_BURGERS, 1, 7000), (npw.NPW_FLUX_ADVECTION, 1, 9000),
                       (npw.NPW_FLUX_EULER1D, 3, 6500), (npw.NPW_FLUX_BURGERS, 1, 300)):
        x = (np.arange(n) + 0.5) / n
        if m == 3:
            rho = 1.0 + 0.2 * np.sin(2 * np.pi * 2 * x) + 0.5 * (x > 0.5)
            f = np.concatenate([rho, 0.1 * rho, 1.0 / 0.4 + 0.005 * rho])
        else:
            f = 1.0 + 0.5 * np.sin(2 * np.pi * x + g.uniform(0, 6))
        specs.append(dict(kind=kind, nx=n, dx=1.0 / n, t_end=0.02, cfl=0.5, bc=0))
        fields.append(f)
        ms.append(m)
    table, total, offs = npw.make_queue_instances(specs)
    for max_steps in (0, 5):
        p = npw.Params(precision=npw.NPW_FP32_MIXED, batch_mode=1, max_steps=max_steps)
        arena = torch.tensor(np.concatenate(fields), dtype=torch.float32, device="cuda")
        st, stats = npw.npweno_queue_solve(arena, table, p, raise_on_error=False)
        assert st == (npw.NPW_ETIMEOUT if max_steps else 0)
        a = arena.cpu().numpy()
        for sp, u0, off, s, m in zip(specs, fields, offs, stats, ms):
            tb, _ = npw.make_instances([sp["nx"]], [sp["dx"]], [sp["t_end"]], [sp["cfl"]], [sp["bc"]], m=m)
            u = torch.tensor(u0, dtype=torch.float32, device="cuda")
            stb, rs = npw.npweno_batch_solve(u, tb, m, sp["kind"], p, raise_on_error=False)
            rs = rs[0]
            assert s["status"] == rs["status"] and s["steps"] == rs["steps"], (sp, s, rs)
            if max_steps:
                assert s["steps"] == max_steps and s["status"] == npw.NPW_ETIMEOUT
            assert np.array_equal(a[off:off + u0.size], u.cpu().numpy()), (sp["kind"], sp["nx"])
