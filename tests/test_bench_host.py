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
