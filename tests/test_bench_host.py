"""Host-side logic of the benchmark that needs no GPU: the serving request stream and the
first-in first-out latency recurrence of the FP64 comparator."""
import numpy as np

import bench


def test_fifo_latencies_queue_recurrence():
    lat, end = bench.fifo_latencies(np.array([1.0, 2.0, 0.5, 0.25]), [0.0, 0.5, 10.0, 10.1])
    # request 1 waits for request 0 (ends at 1.0), request 3 for request 2 (ends at 10.5)
    np.testing.assert_allclose(lat, [1.0, 2.5, 0.5, 0.65])
    assert end == 10.75


def test_serving_stream_is_the_same_requests_at_every_rate():
    a = bench.serving_requests(20, 10.0)
    b = bench.serving_requests(20, 1000.0)
    assert [r["n"] for r in a] == [r["n"] for r in b]
    assert [r["kind"] for r in a] == [r["kind"] for r in b]
    assert all(np.array_equal(x["u0"], y["u0"]) for x, y in zip(a, b))
    # arrival times scale with 1 / rate
    np.testing.assert_allclose([r["arrival"] for r in a], [100.0 * r["arrival"] for r in b], rtol=1e-12)
    assert {r["kind"] for r in a} <= {1, 2, 3}
    for r in a:  # 2D requests are square Euler domains, [4][n][n]
        if r["kind"] == 3:
            assert r["ny"] == r["n"] and r["u0"].shape == (4, r["n"], r["n"]) and r["m"] == 4
        else:
            assert r["ny"] == 0 and r["u0"].size == r["m"] * r["n"]
