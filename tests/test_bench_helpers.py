"""Host logic of the benchmark (no GPU): the recorded ncu traffic is found for the committed
action kernels and dropped when their source changes, the launch count per step, and the
clock sampler's fallback when NVML cannot be loaded."""
import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


def test_recorded_traffic_matches_committed_kernel(bench):
    fp4 = bench.recorded_traffic("action_tc_kernel<1>", "d=4 N=65536 seed 1")
    fp8 = bench.recorded_traffic("action_tc_kernel<0>", "d=4 N=65536 seed 1")
    assert fp4 is not None and fp8 is not None and fp8 > fp4 > 0
    assert bench.recorded_traffic("action_popc_kernel<16, 0>", "d=4 N=65536 seed 1") is not None
    assert bench.recorded_traffic("action_tc_kernel<1>", "d=4 N=40000 seed 1") is None
    assert bench.recorded_traffic("no_such_kernel", "d=4 N=65536 seed 1") is None


def test_recorded_traffic_dropped_when_device_code_changes(bench, tmp_path, monkeypatch):
    import json
    import shutil
    src = os.path.join(ROOT, "paper_1709_03013_gb300", "csrc", "action_tc.cu")
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    fake_root = tmp_path
    (fake_root / "profiles").mkdir()
    (fake_root / "paper_1709_03013_gb300" / "csrc").mkdir(parents=True)
    json.dump(rec, open(fake_root / "profiles" / "traffic.json", "w"))
    dst = fake_root / "paper_1709_03013_gb300" / "csrc" / "action_tc.cu"
    shutil.copy(src, dst)
    monkeypatch.setattr(bench, "ROOT", str(fake_root))
    assert bench.recorded_traffic("action_tc_kernel<1>", "d=4 N=65536 seed 1") is not None
    text = dst.read_text()
    marker = "// ------------------------------------------------------------------ host side"
    i = text.index(marker)
    dst.write_text(text[:i] + "// a comment only\n" + text[i:])          # comments do not count
    assert bench.recorded_traffic("action_tc_kernel<1>", "d=4 N=65536 seed 1") is not None
    dst.write_text(text[:i] + "static int changed_device_code = 1;\n" + text[i:])
    assert bench.recorded_traffic("action_tc_kernel<1>", "d=4 N=65536 seed 1") is None
    # the host code that orders the kernel's tiles counts too (it changes the traffic)
    dst.write_text(text + "\nstatic int changed_host_code = 1;\n")
    assert bench.recorded_traffic("action_tc_kernel<1>", "d=4 N=65536 seed 1") is None


def test_launches_per_step(bench):
    # sprinkle, chunk sort, 6 merge passes, gather, screen values, link, expand, action, finalize
    assert bench.launches_per_step(65536, True) == 14
    assert bench.launches_per_step(65536, False) == 13
    assert bench.launches_per_step(1024, True) == 8


def test_clock_sampler_falls_back_without_nvml(bench, monkeypatch):
    import ctypes
    real = ctypes.CDLL

    def no_nvml(name, *a, **k):
        if "nvidia-ml" in str(name):
            raise OSError("not here")
        return real(name, *a, **k)

    monkeypatch.setattr(ctypes, "CDLL", no_nvml)
    assert isinstance(bench.clock_sampler(0), bench.ClockSampler)
