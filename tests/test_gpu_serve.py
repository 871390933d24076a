"""The continuous-batching server: every result rendered inside a mixed batch
equals the same request rendered alone, the admission budget is respected,
and the one-at-a-time configuration serves in arrival order."""
import numpy as np
import pytest
import torch

from paper_2411_12788_gb300 import raster, scenes, serve

pytestmark = pytest.mark.gpu

SIZES = [(64, 48), (160, 120), (320, 240), (96, 200)]


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_results_same_alone_and_in_mix():
    _need_gpu()
    sc = scenes.cluster_scene(100_000, 64, seed=5, sh_degree=3)
    g = raster.GaussianTensors.from_scene(sc)
    trace = serve.poisson_trace(24, rate=2000.0, seed=7, sizes=SIZES)     # arrivals overlap
    srv = serve.RenderServer(g, budget_bytes=4 << 30, streams=2, max_views=8, keep_images=True)
    srv.serve(trace)
    assert srv.batches_run < len(trace)            # requests were actually batched
    assert len({r.batch for r in trace}) == srv.batches_run
    for r in trace:
        alone = raster.forward(g, [r.cam]).outs["image"]
        mixed = r.image.reshape(-1)
        assert mixed.shape == alone.shape
        assert torch.allclose(mixed, alone, atol=1e-6, rtol=0), r.rid
        assert r.done >= r.arrival


def test_one_at_a_time_is_fifo_and_budget_holds():
    _need_gpu()
    sc = scenes.cluster_scene(50_000, 64, seed=6, sh_degree=0)
    g = raster.GaussianTensors.from_scene(sc)
    trace = serve.poisson_trace(16, rate=500.0, seed=8, sizes=SIZES)
    srv = serve.RenderServer(g, budget_bytes=1 << 30, streams=1, max_views=1)
    srv.serve(trace)
    assert srv.batches_run == len(trace)
    done = [r.done for r in trace]
    assert done == sorted(done)
    # a budget smaller than any single request still serves everything, one by one
    trace = serve.poisson_trace(6, rate=5000.0, seed=9, sizes=SIZES)
    srv = serve.RenderServer(g, budget_bytes=1 << 20, streams=3, max_views=8)
    srv.serve(trace)
    assert all(r.done is not None for r in trace)
    assert srv.batches_run == len(trace)


def test_allocation_failure_propagates_and_server_recovers():
    """Host-side fault injection: the third buffer request of the trace
    fails; the error reaches the caller, the collector is restored, and the
    same server serves the next trace."""
    _need_gpu()
    import gc
    sc = scenes.cluster_scene(50_000, 64, seed=10, sh_degree=0)
    g = raster.GaussianTensors.from_scene(sc)
    srv = serve.RenderServer(g, budget_bytes=1 << 30, streams=2, max_views=4)
    real = srv._buf
    calls = {"n": 0}

    def failing(slot, name, nbytes):
        calls["n"] += 1
        if calls["n"] == 3:
            raise RuntimeError("injected allocation failure")
        return real(slot, name, nbytes)
    srv._buf = failing
    with pytest.raises(RuntimeError, match="injected"):
        srv.serve(serve.poisson_trace(8, rate=5000.0, seed=11, sizes=SIZES))
    assert gc.isenabled()
    srv._buf = real
    torch.cuda.synchronize()
    srv.reserved = 0
    trace = serve.poisson_trace(8, rate=5000.0, seed=12, sizes=SIZES)
    srv.serve(trace)
    assert all(r.done is not None for r in trace)


def test_cancelled_requests_are_dropped():
    """Requests cancelled before admission (host-side fault injection of a
    client that gives up) are never rendered and leave no completion; the
    rest of the trace is served and the statistics count only them."""
    _need_gpu()
    sc = scenes.cluster_scene(50_000, 64, seed=13, sh_degree=0)
    g = raster.GaussianTensors.from_scene(sc)
    trace = serve.poisson_trace(15, rate=3000.0, seed=14, sizes=SIZES)
    for r in trace[::3]:
        r.cancelled = True
    srv = serve.RenderServer(g, budget_bytes=1 << 30, streams=2, max_views=4)
    srv.serve(trace)
    for r in trace:
        if r.cancelled:
            assert r.done is None and r.batch == -1
        else:
            assert r.done is not None and r.done >= r.arrival
    assert srv.views_run == len(trace) - len(trace[::3])
    assert serve.latency_stats(trace)["requests"] == len(trace) - len(trace[::3])

