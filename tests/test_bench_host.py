"""Host logic of bench.py's measurement contract, on CPU: the clock record
taken during the timed region (median SM clock, max clock, throttle reasons
seen), the whole-job throughput, the peak used as the roofline denominator,
and the rule that a committed DRAM-traffic figure is reported only while the
kernel source it was taken on is unchanged."""

import json
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _DoneProc:
    """Stands in for the finished nvidia-smi process."""

    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.proc = _DoneProc()
    s.lines = list(lines)
    return s


def test_clock_record_median_max_and_reasons():
    lines = [
        "2070, 2070, 900.5, Not Active, Not Active, Not Active, Not Active",
        "2055, 2070, 1300.0, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 1350.2, Not Active, Not Active, Not Active, Active",
        "1980, 2070, 1390.0, Active, Not Active, Not Active, Not Active",
        "garbage line",
        "[N/A], 2070, 10, Not Active, Not Active, Not Active, Not Active",
    ]
    rec = _sampler(lines).stop()
    assert rec["samples"] == 4
    assert rec["sm_mhz"] == pytest.approx(2062.5)  # median of 2070, 2055, 2070, 1980
    assert rec["sm_max_mhz"] == 2070
    assert rec["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_clock_record_without_samples_or_tool():
    rec = _sampler([]).stop()
    assert rec["sm_mhz"] is None and rec["samples"] == 0 and rec["reasons"] == []
    s = bench.ClockSampler(0)  # never started: no nvidia-smi
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_whole_job_throughput_counts_every_rank_over_the_slowest_time():
    # one rank: 8 GB in 1 s
    assert bench.aggregate(8e9, 1000.0, 1) == pytest.approx(8.0)
    # four replicas, the slowest took 2 s: 4 x 8 GB / 2 s
    assert bench.aggregate(8e9, 2000.0, 4) == pytest.approx(16.0)
    assert bench.reduce_max(3.5, 1) == 3.5


def _fake_root(tmp_path):
    csrc = tmp_path / "paper_2405_01250_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in ("apply.cu", "common.cuh"):
        shutil.copy(os.path.join(ROOT, "paper_2405_01250_gb300", "csrc", f), csrc / f)
    (tmp_path / "profiles").mkdir()
    return tmp_path


def test_traffic_reported_only_for_the_source_it_was_taken_on(tmp_path, monkeypatch):
    root = _fake_root(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench._traffic("cp_c128") is None  # no record at all
    h = bench._kernel_source_hash()
    rec = {"cp_c128": {"bytes_per_launch": 8.3e9, "source_hash": h}}
    (root / "profiles" / "dram_traffic.json").write_text(json.dumps(rec))
    assert bench._traffic("cp_c128") == 8.3e9
    assert bench._traffic("other_kernel") is None
    # any change to the kernel source invalidates the figure
    with open(root / "paper_2405_01250_gb300" / "csrc" / "apply.cu", "a") as f:
        f.write("\n// edited\n")
    assert bench._kernel_source_hash() != h
    assert bench._traffic("cp_c128") is None


def test_committed_traffic_record_is_well_formed():
    with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
        d = json.load(f)
    e = d["cp_c128"]
    assert len(e["source_hash"]) == 16
    # traffic is a DRAM measurement of one 28-qubit launch: close to, and not
    # far above, the algorithmic 2 x 2^28 x 16 bytes
    alg = 2 * (1 << 28) * 16
    assert 0.9 * alg <= e["bytes_per_launch"] <= 1.1 * alg
    assert os.path.exists(os.path.join(ROOT, e["profile"]))


def test_peak_is_measured_when_present_else_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6779.0, "bf16_tflops": 1900.0}))
    assert bench._peaks() == (6779.0, "measured")


def test_reference_arm_reports_the_same_config_as_the_gpu_arm():
    """The oracle arm runs a bounded sample of the same QFT workload and
    prints the GPU arm's config (both come from qft_config); its sampling is
    stated in cpu_baseline."""
    import argparse

    import synth
    args = argparse.Namespace(qubits=10, ref_gates=3, steps=1, warmup=0)
    line = bench.run_reference(args, 0, 1)
    circ, _ = synth.qft(10, seed=0)
    assert line["config"] == bench.qft_config(10, len(circ.gates), 1)
    assert line["config"]["ops_per_step"] == 10 + 45 + 5
    assert line["impl"] == "reference" and line["unit"] == bench.UNIT and line["higher_is_better"]
    assert line["cpu_baseline"]["kind"] == "oracle" and "3 of the 60" in line["cpu_baseline"]["sample"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert bench.qft_config(28, 420, 1)["l2"] == "inputs larger than L2 (4 GiB state vs 129 MB L2); no flush"
    assert bench.qft_config(28, 420, 4)["parallelism"] == "replicas"


def test_gpus_flag_must_match_the_launched_ranks():
    """bench.py --gpus N runs one rank per GPU: without N ranks (WORLD_SIZE)
    it refuses, before any GPU work, instead of reporting one replica."""
    import subprocess
    env = dict(os.environ)
    env.pop("WORLD_SIZE", None)
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "4", "--steps", "1"],
                       capture_output=True, text=True, env=env, timeout=120)
    assert p.returncode == 2 and "needs 4 ranks" in p.stderr
    env["WORLD_SIZE"] = "2"
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "1", "--impl", "reference"],
                       capture_output=True, text=True, env=env, timeout=120)
    assert p.returncode == 2 and "WORLD_SIZE is 2" in p.stderr


def test_precision_fields_helpers():
    """The bench's state comparison and complex64 bound agree with the test
    suite's (gpu_util) and with the oracle's error measures."""
    import numpy as np
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import gpu_util
    import oracle
    ks = [1, 0, 2, 3, 1, 0]
    assert bench._c64_bound(ks) == pytest.approx(gpu_util.c64_circuit_bound(ks), rel=1e-15)
    rng = np.random.default_rng(0)
    a = rng.standard_normal(64) + 1j * rng.standard_normal(64)
    b = a + 1e-6 * (rng.standard_normal(64) + 1j * rng.standard_normal(64))
    e = bench.state_errors(b, a)
    assert e["fidelity_vs_oracle"] == pytest.approx(oracle.fidelity(a, b), rel=1e-14)
    assert e["max_abs_err_vs_oracle"] == oracle.max_abs_err(a, b)


def test_fp64_floor_model_counts():
    """The FP64-instruction model behind the adjoint and batch floors, on a
    hand-countable circuit: a fixed gate before the first rotation counts
    forward only; rotations take 2 forward / 6 reverse scaled (4 / 10
    unscaled); a fixed gate after it 4 / 8; chunk-form runs (blocks of 256,
    the higher chunks' product once per block) p + 4 forward and p + 12 + v/8
    reverse with p = 4 + 4 (c - 2) / 8; weight-form runs 4 / 11; lambda 2
    per real group with equal weights, 2 more per further chunk of 8 terms
    when they differ, plus 2 for the energy."""
    import numpy as np
    import synth
    g = [synth.Gate((0,), synth.H),                                   # before the first rotation
         synth.Gate((1,), None, param=0, gen="X"),
         synth.Gate((0, 1), synth.CZ),                                # a sign gate: no FP64 work
         synth.Gate((1,), synth.random_gate(1, np.random.default_rng(0), "dense")),
         synth.Gate((0, 1), None, param=1, gen="ZZ")]                 # a Z-type rotation
    obs = synth.Observable(np.array([0, 0, 1], dtype=np.uint64), np.array([3, 1, 0], dtype=np.uint64),
                           np.array([1.0, 1.0, 0.5]))
    # lambda: group x=0 (two terms, equal) 2, group x=1 (one term) 2, energy 2
    assert bench.fp64_per_amp(g, obs, runs=False) == (4 + 4 + 4 + 4, 10 + 8 + 10, 6)
    assert bench.fp64_per_amp(g, obs, runs=False, scaled=True) == (4 + 2 + 4 + 2, 6 + 8 + 6, 6)
    # with runs the Z-type rotation and the sign gate move into the runs given
    f, r, lam = bench.fp64_per_amp(g, obs, runs=True, chunks_run=[(0, 0)], scaled=True)
    assert (f, r, lam) == (4 + 2 + 4 + 4, 6 + 8 + 11, 6)
    f, r, _ = bench.fp64_per_amp(g, obs, runs=True, chunks_run=[(8, 3)], scaled=True)
    p = 4 + 4 * 1 / 8
    assert (f, r) == (4 + 2 + 4 + p + 4, 6 + 8 + p + 12 + 8 / 8)
    # unequal weights in one group of 9 terms: two chunks of 8
    obs9 = synth.Observable(np.zeros(9, dtype=np.uint64), np.arange(1, 10, dtype=np.uint64),
                            np.linspace(0.1, 0.9, 9))
    assert bench.fp64_per_amp(g, obs9, runs=False)[2] == 2 + 2 + 2
