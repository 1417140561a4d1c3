"""CPU checks of bench.py's host-side helpers (no GPU)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _peaks(idx, power):
    dt = np.dtype([("idx", "<i8"), ("power", "<f8"), ("freq", "<f8"), ("period", "<f8"), ("flags", "<i4"),
                   ("reserved", "<i4")])
    a = np.zeros(len(idx), dtype=dt)
    a["idx"] = idx
    a["power"] = power
    return a


def test_parity_vs_oracle_batch_top1_and_top3():
    import bench
    ref = {"kind": "batch", "objects": np.array([0, 2]), "arg_idx": np.array([10, 20]),
           "arg_pow": np.array([0.5, 0.25])}
    got = bench.parity_vs_oracle(ref, _peaks([10, 99, 22], [0.50001, 0.1, 0.25]), 1)
    assert got["argmax_within_1_bin"] == 0.5 and got["argmax_exact"] == 0.5
    assert abs(got["max_abs_err_peak_power"] - 1e-5) < 1e-12
    # top-3 rows: only each object's first entry is its maximum
    pk = _peaks([10, 3, 4, 0, 0, 0, 21, 5, 6], [0.5, 0.4, 0.3, 0, 0, 0, 0.25, 0.2, 0.1])
    got = bench.parity_vs_oracle(ref, pk, 3)
    assert got["argmax_within_1_bin"] == 1.0 and got["argmax_exact"] == 0.5


def test_parity_vs_oracle_single_object():
    import bench
    ref = {"kind": "single", "k": np.array([1, 3]), "power": np.array([0.2, 0.4])}
    power = np.array([0.0, 0.2 + 3e-5, 0.0, 0.4], dtype=np.float32)
    got = bench.parity_vs_oracle(ref, None, 1, power)
    assert got["within"] and abs(got["max_abs_err"] - 3e-5) < 1e-6
    assert bench.parity_vs_oracle(None, None, 1) is None


def test_reference_arm_prints_the_contract_line():
    # the reference arm runs the CPU oracle only: its JSON line is checkable here
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["config"]["workload"] == "ragged_lognormal"  # the largest batch is the default


def test_warmup_below_three_is_refused():
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--warmup", "1"],
                         capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert out.returncode != 0 and "warmup" in out.stderr


def test_clock_sampler_waits_for_the_first_sample(monkeypatch):
    """The timed region starts only after nvidia-smi has printed its first row,
    and the summary takes the rows inside the marked region."""
    import io
    import subprocess
    import threading
    import time
    import bench

    release = threading.Event()
    row = "0, 2070, 2070, 500.0, 0x0, Not Active, Not Active, Not Active, Active\n"

    class SlowOut(io.TextIOBase):
        def __init__(self):
            self.n = 0

        def __iter__(self):
            return self

        def __next__(self):
            if self.n == 0:
                release.wait(5.0)  # start-up: nothing printed yet
            if self.n >= 6:
                raise StopIteration
            self.n += 1
            time.sleep(0.02)
            return row

    class FakeProc:
        def __init__(self, *a, **k):
            self.stdout = SlowOut()

        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

        def kill(self):
            pass

    monkeypatch.setattr(subprocess, "Popen", FakeProc)
    clk = bench.ClockSampler("0")
    threading.Timer(0.5, release.set).start()
    t0 = time.time()
    clk.start()
    assert time.time() - t0 >= 0.5  # returned only after the first row
    clk.mark(0)
    time.sleep(0.2)
    clk.mark(1)
    got = clk.stop()
    assert got["sm_mhz"] == 2070.0 and got["sm_max_mhz"] == 2070.0
    assert got["reasons"] == ["sw_power_cap"] and got["power_w_max"] == 500.0


def test_mlp_mode_has_no_reference_arm():
    # --mlp times the library's tensor-core GEMMs; its reference arm says so in one JSON line
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--mlp", "--impl", "reference"],
                         capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and "unavailable" in line
