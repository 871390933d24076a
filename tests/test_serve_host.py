"""Host-side pieces of the server that need no GPU: the Poisson trace and
the latency statistics; scene checkpoints."""
import numpy as np

from paper_2411_12788_gb300 import scenes, serve


def test_poisson_trace_rate_and_sizes():
    tr = serve.poisson_trace(4000, rate=200.0, seed=3)
    t = np.array([r.arrival for r in tr])
    assert np.all(np.diff(t) > 0)
    assert abs(len(t) / t[-1] - 200.0) < 12.0
    sizes = {(r.cam.width, r.cam.height) for r in tr}
    assert sizes == {(640, 480), (1280, 720), (1920, 1080), (3840, 2160)}
    radii = np.array([np.linalg.norm(-r.cam.R.T @ r.cam.t) for r in tr])
    assert radii.min() >= 3.0 and radii.max() <= 6.0


def test_latency_stats():
    tr = serve.poisson_trace(200, rate=100.0, seed=1)
    for k, r in enumerate(tr):
        r.done = r.arrival + (0.001 if k % 100 else 0.050)
    st = serve.latency_stats(tr, skip=0)
    assert abs(st["p50_ms"] - 1.0) < 1e-6
    assert st["max_ms"] > 49.9 and st["requests"] == 200


def test_latency_stats_split_wait_and_service():
    """With launch start times recorded, the slowest request's latency splits
    into the wait before its batch began and the service after it."""
    tr = serve.poisson_trace(100, rate=100.0, seed=2)
    for k, r in enumerate(tr):
        r.started = r.arrival + (0.030 if k == 50 else 0.0002)
        r.done = r.started + 0.001
    st = serve.latency_stats(tr)
    assert abs(st["max_ms"] - 31.0) < 1e-6
    assert abs(st["slowest_wait_ms"] - 30.0) < 1e-6 and abs(st["slowest_service_ms"] - 1.0) < 1e-6
    assert abs(st["service_p99_ms"] - 1.0) < 1e-6
    # without start times there is no split
    assert "wait_p99_ms" not in serve.latency_stats([serve.Request(0, 0.0, tr[0].cam, done=0.001)])


def test_scene_save_load_round_trip(tmp_path):
    """A scene written with Scene.save reads back bit-identical."""
    sc = scenes.cluster_scene(500, 8, seed=2, sh_degree=3)
    path = tmp_path / "scene.npz"
    sc.save(path)
    back = scenes.load(path)
    assert back.sh_degree == sc.sh_degree
    for k in ("means", "scales", "rotations", "opacities", "sh"):
        a, b = getattr(sc, k), getattr(back, k)
        assert a.dtype == b.dtype and np.array_equal(a, b), k


def test_latency_stats_leave_out_cancelled_requests():
    tr = serve.poisson_trace(10, rate=100.0, seed=4)
    for k, r in enumerate(tr):
        if k % 2:
            r.cancelled = True
        else:
            r.done = r.arrival + 0.001 * (k + 1)
    st = serve.latency_stats(tr)
    assert st["requests"] == 5
    assert abs(st["max_ms"] - 9.0) < 1e-9

