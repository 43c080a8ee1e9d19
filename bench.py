"""Benchmark of the DiaQ gate-apply path on GB300.

One step = the QFT of a seeded basis state on 28 qubits in complex128
(420 DiaQ ops: 28 H, 378 controlled phases, 14 SWAPs, applied out of place
by the on-the-fly DiaQ SpMV) followed by the FP64 norm. The metric is the
algorithmic HBM throughput of the gate apply: every op reads the 4 GiB state
and writes the 4 GiB result (2 * 2^28 * 16 bytes), the norm reads it once.
The state (4 GiB) is 32x larger than L2, so no flush is needed between steps.

Prints one JSON line (rank 0). Under torchrun (N > 1) each rank runs an
independent replica (the circuit is not sharded); `value` is the sum of the
ranks' work over the slowest rank's time.

`--impl reference` times the FP64 CPU oracle on the host cores instead (a
bounded sample of the same circuit's gates per step).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DiaQ gate-apply HBM GB/s vs ~8 TB/s at 28-30q; adjoint grads/s vs plain"
UNIT = "GB/s"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def _dist():
    import torch.distributed as dist
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1 and not dist.is_initialized():
        backend = "nccl" if os.environ.get("DIAQ_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend=backend)
    return (dist.get_rank() if ws > 1 else 0), ws


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("apply.cu", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2405_01250_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kernel)
    if not e or e.get("source_hash") != _kernel_source_hash():
        return None
    return e.get("bytes_per_launch")


def _qft_ops(api, circ, n, variant):
    return [api.build(g, n, variant=variant) for g in circ.gates]


def run_ours(args, rank, world):
    import torch
    import torch.distributed as dist
    from paper_2405_01250_gb300 import build as B
    if rank == 0 or not os.path.exists(B.LIB):
        B.build()
    if world > 1:
        dist.barrier()
    from paper_2405_01250_gb300 import api
    import synth

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    n = args.qubits
    N = 1 << n
    circ, j = synth.qft(n, seed=0)
    ops = _qft_ops(api, circ, n, "onthefly")
    classes = [op.info()["class"] for op in ops]
    stream = torch.cuda.current_stream()
    x0 = torch.zeros(N, dtype=torch.complex128, device="cuda")
    x0[j] = 1.0
    a = x0.clone()
    b = torch.empty_like(a)
    assert len(ops) % 2 == 0
    bytes_op = 2 * N * 16
    bytes_step = len(ops) * bytes_op + N * 16

    def step(record=None):
        x, y = a, b  # an even op count leaves the state in `a` again
        if record is not None:
            record[0].record(stream)
        for i, op in enumerate(ops):
            api.apply(op, x, y)
            if record is not None:
                record[i + 1].record(stream)
            x, y = y, x
        return api.norm(x)

    for _ in range(args.warmup):
        nrm = step()
    assert abs(nrm - 1.0) < 1e-10, f"norm {nrm}"
    # timed region
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(ops) + 1)] for _ in range(args.steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    t0.record(stream)
    for s in range(args.steps):
        step(ev[s])
    t1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    if world > 1:
        dist.barrier()
    ms_total = t0.elapsed_time(t1)
    # per-op durations by class
    dur = {}
    for s in range(args.steps):
        for i, c in enumerate(classes):
            dur.setdefault(c, []).append(ev[s][i].elapsed_time(ev[s][i + 1]))
    apply_ms = sum(sum(v) for v in dur.values()) / args.steps
    if world > 1:
        t = torch.tensor([ms_total], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    ms_step = ms_total / args.steps
    value = world * bytes_step * args.steps / (ms_total / 1e3) / 1e9

    # dominant kernel: controlled phase (diagonal class) launches
    dom = "diagonal"
    dom_ms = statistics.mean(dur[dom])
    peak, peak_kind = _peaks()
    achieved = bytes_op / (dom_ms / 1e3) / 1e9
    per_class = {c: {"launches_per_step": len(v) // args.steps, "mean_ms": statistics.mean(v),
                     "gbs": bytes_op / (statistics.mean(v) / 1e3) / 1e9} for c, v in dur.items()}

    # end to end through diaq_simulate: pinned host |j> in, pinned host result out
    e2e = None
    if not args.no_e2e:
        hin = torch.zeros(N, dtype=torch.complex128, pin_memory=True)
        hin[j] = 1.0
        hout = torch.empty(N, dtype=torch.complex128, pin_memory=True)
        w0 = torch.empty_like(a)
        api.simulate(ops, hin, hout, w0)  # warm
        torch.cuda.synchronize()
        te = time.perf_counter()
        e_steps = max(1, min(args.steps, 3))
        for _ in range(e_steps):
            api.simulate(ops, hin, hout, w0)
        e_s = (time.perf_counter() - te) / e_steps
        amp_ok = abs(complex(hout[0]) - 1 / math.sqrt(N)) < 1e-12
        e2e = {"value": world * len(ops) * bytes_op / e_s / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": N * 16, "d2h_bytes_per_step": N * 16, "ms_per_step": e_s * 1e3,
               "api": "diaq_simulate (in-place on-the-fly ops, pinned host buffers)", "checked": bool(amp_ok)}
        del hin, hout, w0

    # stored-diagonal variant: a sample of ops materialised and applied
    stored = None
    if not args.no_stored:
        sample = [circ.gates[0], circ.gates[1], circ.gates[-1]]  # H, CP, SWAP
        res = {}
        for g in sample:
            t_b0 = torch.cuda.Event(enable_timing=True)
            t_b1 = torch.cuda.Event(enable_timing=True)
            t_b0.record(stream)
            op = api.build(g, n, variant="stored")
            t_b1.record(stream)
            info = op.info()
            for _ in range(2):
                api.apply(op, a, b)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            reps = 3
            e0.record(stream)
            for _ in range(reps):
                api.apply(op, a, b)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            alg = 2 * N * 16 + info["stored_bytes"]
            res[g.name] = {"apply_ms": ms, "gbs": alg / (ms / 1e3) / 1e9, "stored_bytes": info["stored_bytes"],
                           "build_ms": t_b0.elapsed_time(t_b1)}
            op.close()
        stored = res

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128 (f64 arithmetic)", "data": "synthetic",
        "config": {"workload": f"qft-{n} complex128, on-the-fly DiaQ apply of {len(ops)} ops + FP64 norm",
                   "qubits": n, "ops_per_step": len(ops), "state_bytes": N * 16,
                   "l2": "inputs larger than L2 (4 GiB state vs 129 MB L2); no flush", "parallelism":
                   "replicas" if world > 1 else "single GPU"},
        "gates_per_s": world * len(ops) * args.steps / (ms_total / 1e3),
        "apply_only_gbs": len(ops) * bytes_op / (apply_ms / 1e3) / 1e9,
        "per_class": per_class,
        "roofline": {"bound": "hbm", "kernel": "k_apply_small<double,2,1> (controlled phase, diagonal class)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": f"{peak_kind} hbm_gbs", "traffic": _traffic("cp_c128")},
        "e2e": e2e, "stored": stored, "clocks": clocks,
        "gpu_launches": args.steps * (len(ops) + 2),
    }
    if rank == 0 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(n, circ, j, budget_s=args.cpu_seconds)
    return out


def cpu_baseline(n, circ, j, budget_s=12.0):
    """The FP64 oracle (as it stands) on the host cores, on a bounded sample
    of the same circuit's gates: GB/s of algorithmic gate-apply bytes."""
    import oracle
    import synth  # noqa: F401
    N = 1 << n
    x = np.zeros(N, dtype=np.complex128)
    x[j] = 1.0
    t0 = time.perf_counter()
    done = 0
    for g in circ.gates:
        x = oracle.apply_gate(x, g.targets, g.matrix)
        done += 1
        if time.perf_counter() - t0 > budget_s and done >= 2:
            break
    el = time.perf_counter() - t0
    return {"value": done * 2 * N * 16 / el / 1e9, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": f"first {done} of {len(circ.gates)} ops of qft-{n} (complex128), {el:.1f} s"}


def run_reference(args, rank, world):
    """FP64 CPU oracle as the reference arm: each step applies a bounded
    sample of the QFT gates on the host cores."""
    import oracle
    import synth
    n = args.qubits
    N = 1 << n
    circ, j = synth.qft(n, seed=0)
    per_step = max(1, args.ref_gates)
    x = np.zeros(N, dtype=np.complex128)
    x[j] = 1.0
    gi = 0

    def step():
        nonlocal x, gi
        for _ in range(per_step):
            g = circ.gates[gi % len(circ.gates)]
            x = oracle.apply_gate(x, g.targets, g.matrix)
            gi += 1

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = time.perf_counter() - t0
    value = args.steps * per_step * 2 * N * 16 / el / 1e9
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128 (f64 arithmetic)", "data": "synthetic",
        "config": {"workload": f"qft-{n} complex128, FP64 CPU oracle, {per_step} ops per step", "qubits": n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                         "sample": f"{per_step} qft-{n} ops per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--qubits", type=int, default=28)
    ap.add_argument("--ref-gates", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-stored", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        world = int(os.environ.get("WORLD_SIZE", "1"))
        if rank != 0:
            return
        print(json.dumps(run_reference(args, rank, world)), flush=True)
        return
    rank, world = _dist()
    out = run_ours(args, rank, world)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
