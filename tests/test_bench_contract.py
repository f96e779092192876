"""The reference arm's JSON line (bench.py --impl reference) on the CPU, with the oracle's timed
sample replaced by a fixed stand-in: the keys the benchmark contract asks for, the whole-job
step definition (one step = every frequency of the workload) and the zero host-device traffic
of a CPU arm."""
import argparse
import json

import bench


def test_reference_line_keys_and_step(monkeypatch, capsys):
    monkeypatch.setattr(bench, "oracle_sample", lambda: (0.01, "stand-in sample", 0.5))
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    bench.run_reference(argparse.Namespace(warmup=3, steps=2, gpus=1))
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "e2e",
                "cpu_baseline"):
        assert key in line, key
    assert line["impl"] == "reference" and line["unit"] == "solves/s"
    assert line["value"] == 0.01
    assert abs(line["ms_per_step"] - 1e3 * bench.N_FREQ / 0.01) < 1e-6
    assert line["e2e"] == {"value": 0.01, "unit": "solves/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["config"]["workload"].startswith("pressurised spherical cavity")


def test_reference_arm_other_ranks_print_nothing(monkeypatch, capsys):
    monkeypatch.setattr(bench, "oracle_sample", lambda: (0.01, "stand-in sample", 0.5))
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(argparse.Namespace(warmup=3, steps=2, gpus=2))
    assert capsys.readouterr().out == ""


def test_command_line_parses():
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    p = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--help"], capture_output=True, text=True)
    assert p.returncode == 0, p.stderr
    for opt in ("--gpus", "--steps", "--warmup", "--impl", "--workload", "--afs-tol"):
        assert opt in p.stdout


def test_every_side_workload_returns_without_running_the_benchmark(monkeypatch):
    import sys
    calls = []
    for name in ("kernel_case", "kernel_case_single", "profile_step", "hm_kernel_case", "workload_uneven",
                 "workload_porous_afs", "workload_example3", "workload_large", "run_gpu", "run_reference"):
        monkeypatch.setattr(bench, name, lambda *a, _n=name, **k: calls.append(_n))
    flags = [["--kernel-case"], ["--kernel-case-single"], ["--profile-step"], ["--hm-kernel-case"]]
    flags += [["--workload", w] for w in ("uneven", "porous-afs", "porous-afs-full", "example3", "example3-mlp",
                                          "large", "large-hmatrix", "porous-afs-lowband",
                                          "porous-afs-full-lowband", "example3-lowband")]
    for f in flags:
        calls.clear()
        monkeypatch.setattr(sys, "argv", ["bench.py", *f])
        bench.main()
        assert len(calls) == 1 and calls[0] not in ("run_gpu", "run_reference"), (f, calls)
    calls.clear()
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    bench.main()
    assert calls == ["run_gpu"]
