"""Tile sizes of the 1D per-stage kernels and their autotuner: every tiling gives the same
bits (each face gets the same arithmetic whatever CTA computes it), and the tuned size is one
of the candidates and is used by later runs."""
import numpy as np
import pytest

from paper_1602_00182_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TILES = (256, 512, 1024, 2048)


@pytest.fixture(scope="module")
def npw():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1602_00182_gb300 import build as b
    b.build()
    import paper_1602_00182_gb300.npweno as m
    m.load()
    return m


def _burgers_batch(npw, params):
    inst = I.burgers_batch(count=9, nmin=100, nmax=5000, t_end=0.3, seed_index=41)
    ns = [it.n for it in inst]
    table, _ = npw.make_instances(ns, [it.dx for it in inst], [0.3] * len(ns), [0.5] * len(ns), [0] * len(ns))
    dt = torch.float32 if params.precision == 1 else torch.float64
    arena = torch.tensor(np.concatenate([it.u0[0] for it in inst]), dtype=dt, device="cuda")
    st, stats = npw.npweno_batch_solve(arena, table, 1, npw.NPW_FLUX_BURGERS, params)
    assert st == 0
    return arena.cpu().numpy(), [s["steps"] for s in stats]


@pytest.mark.parametrize("precision", [0, 1])
def test_tile_size_does_not_change_results(npw, precision):
    ref = None
    for tile in TILES:
        p = npw.Params(rbf=npw.NPW_RBF_GA, precision=precision, batch_mode=1, tile_1d=tile)
        got, steps = _burgers_batch(npw, p)
        if ref is None:
            ref = (got, steps)
        else:
            assert steps == ref[1]
            assert np.array_equal(got, ref[0]), tile


def test_tile_size_euler_characteristic(npw):
    it = I.euler_batch(count=2, nmin=3000, nmax=3100, seed_index=42)[1]
    out = []
    for tile in (256, 2048):
        u = torch.tensor(it.u0, dtype=torch.float32, device="cuda")
        p = npw.Params(precision=1, characteristic=1, tile_1d=tile)
        st = npw.npweno_solve(u, it.dx, 0.05 * it.t_end, 0.5, npw.NPW_FLUX_EULER1D, 1, p)
        assert st["status"] == 0
        out.append(u.cpu().numpy())
    assert np.array_equal(out[0], out[1])


def test_autotune_picks_a_candidate_used_by_later_runs(npw):
    p0 = npw.Params(rbf=npw.NPW_RBF_GA, precision=1, batch_mode=1)
    best = npw.npw_autotune_1d(npw.NPW_FLUX_BURGERS, 1, p0)
    assert best in TILES
    tuned, s1 = _burgers_batch(npw, p0)  # tile_1d = 0: the tuned size
    fixed, s2 = _burgers_batch(npw, npw.Params(rbf=npw.NPW_RBF_GA, precision=1, batch_mode=1, tile_1d=1024))
    assert s1 == s2 and np.array_equal(tuned, fixed)
    assert npw.npw_autotune_1d(npw.NPW_FLUX_EULER1D, 3, npw.Params(precision=0)) in TILES
