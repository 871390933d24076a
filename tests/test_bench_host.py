"""Host-side checks of bench.py: every leg the default run calls exists and
the argument parser accepts the documented flags (no GPU needed)."""
import importlib
import sys

import pytest


def test_bench_defines_every_leg():
    bench = importlib.import_module("bench")
    for name in ("run_ours", "run_e2e", "run_serving", "run_dense", "run_culling", "run_strategies",
                 "cpu_baseline", "run_reference", "roofline", "kernel_times", "main"):
        assert callable(getattr(bench, name, None)), name


@pytest.mark.parametrize("argv", [[], ["--gpus", "1", "--steps", "5", "--warmup", "3"],
                                  ["--impl", "reference"], ["--no-e2e", "--no-serve", "--no-dense", "--no-culling",
                                                            "--no-cpu-baseline"]])
def test_bench_parses_flags(argv, monkeypatch):
    bench = importlib.import_module("bench")
    monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
    args = bench.parse()
    assert args.warmup >= 3 and args.steps >= 1


def test_traffic_is_reported_only_for_the_profiled_kernel_and_workload(monkeypatch):
    """The ncu DRAM bytes the roofline carries belong to one build of the
    kernel's source (its SHA-256) and one workload (its entry count): any
    other source or entry count reports no traffic."""
    bench = importlib.import_module("bench")
    rec = dict(bench.PROFILED_TRAFFIC["render_bwd"])
    ok = bench.profiled_traffic("render_bwd", rec["entries"])
    assert ok is None or ok == rec["bytes"]        # None once the source has changed since the capture
    assert bench.profiled_traffic("render_bwd", rec["entries"] + 1) is None
    assert bench.profiled_traffic("render_fwd", rec["entries"]) is None
    monkeypatch.setitem(bench.PROFILED_TRAFFIC, "render_bwd", dict(rec, sha256="0" * 64))
    assert bench.profiled_traffic("render_bwd", rec["entries"]) is None
    monkeypatch.setitem(bench.PROFILED_TRAFFIC, "render_bwd", dict(rec, source="no/such/file.cu"))
    assert bench.profiled_traffic("render_bwd", rec["entries"]) is None
