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


def reduce_max(value: float, world: int) -> float:
    """Max over ranks of a host scalar (the slowest rank's time); gloo
    reduces CPU tensors, NCCL device tensors."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def qft_config(n: int, n_ops: int, world: int) -> dict:
    """The workload both arms report: one step is the QFT-n circuit's n_ops
    DiaQ ops in complex128 plus the FP64 norm (the reference arm times a
    bounded sample of those ops per step and says so in its cpu_baseline)."""
    state = (1 << n) * 16
    return {"workload": f"qft-{n} complex128, on-the-fly DiaQ apply of {n_ops} ops + FP64 norm",
            "qubits": n, "ops_per_step": n_ops, "state_bytes": state,
            "l2": f"inputs larger than L2 ({state / 2**30:g} GiB state vs 129 MB L2); no flush",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def aggregate(bytes_per_rank: float, ms_max: float, world: int) -> float:
    """Whole-job GB/s: every rank runs the same replica, so the units
    processed are world x one rank's, over the slowest rank's time."""
    return world * bytes_per_rank / (ms_max / 1e3) / 1e9


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
    ms_total = reduce_max(ms_total, world)
    ms_step = ms_total / args.steps
    value = aggregate(bytes_step * args.steps, ms_total, world)

    # dominant kernel: controlled phase (diagonal class) launches
    dom = "diagonal"
    dom_ms = statistics.mean(dur[dom])
    peak, peak_kind = _peaks()
    achieved = bytes_op / (dom_ms / 1e3) / 1e9
    per_class = {c: {"launches_per_step": len(v) // args.steps, "mean_ms": statistics.mean(v),
                     "gbs": bytes_op / (statistics.mean(v) / 1e3) / 1e9} for c, v in dur.items()}

    # in place: the same 420 ops with the identity-row skip (a controlled
    # phase reads and writes a quarter of the rows, a SWAP half, H all);
    # bytes counted per op as the path moves them
    inplace_bytes = sum(op.apply_bytes(in_place=True) for op in ops)
    inplace = None
    if not args.no_inplace:
        c = a.clone()
        for _ in range(2):
            for op in ops:
                api.apply(op, c, c)
        i0 = torch.cuda.Event(enable_timing=True)
        i1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        i0.record(stream)
        for _ in range(args.steps):
            for op in ops:
                api.apply(op, c, c)
        i1.record(stream)
        torch.cuda.synchronize()
        ims = i0.elapsed_time(i1) / args.steps
        inplace = {"workload": f"qft-{n} complex128, {len(ops)} ops in place (identity rows skipped)",
                   "ms_per_step": ims, "gates_per_s": len(ops) / (ims / 1e3),
                   "bytes_per_step": inplace_bytes, "gbs": inplace_bytes / (ims / 1e3) / 1e9,
                   "speedup_vs_out_of_place_step": apply_ms / ims, "norm": api.norm(c)}
        del c

    # the same circuit with each run of controlled phases fused into one
    # diagonal op (plan_fusion_diagonal: 28 H, 87 phase runs, 14 SWAPs), in
    # place; gates_per_s counts the circuit's 420 gates
    fused = None
    if not args.no_fused:
        fops = api.build_fused(circ.gates, n, 6, 64, diagonal=True)
        fbytes = sum(op.apply_bytes(in_place=True) for op in fops)
        c = a.clone()
        for _ in range(2):
            for op in fops:
                api.apply(op, c, c)
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        f0.record(stream)
        for _ in range(args.steps):
            for op in fops:
                api.apply(op, c, c)
        f1.record(stream)
        torch.cuda.synchronize()
        fms = f0.elapsed_time(f1) / args.steps
        # the same ops through diaq_simulate in place on the device state
        # (consecutive fused ops merge into passes of up to 11 qubits; H in
        # the scaled form)
        sbytes = api.simulate_bytes(fops)
        api.simulate(fops, c, c, c)
        torch.cuda.synchronize()
        f0.record(stream)
        for _ in range(args.steps):
            api.simulate(fops, c, c, c)
        f1.record(stream)
        torch.cuda.synchronize()
        sms = f0.elapsed_time(f1) / args.steps
        fused = {"workload": f"qft-{n} complex128, runs of controlled phases fused into diagonal ops, in place",
                 "ops": len(fops), "gates": len(ops), "ms_per_step": fms, "gates_per_s": len(ops) / (fms / 1e3),
                 "moved_bytes_per_step": fbytes, "moved_gbs": fbytes / (fms / 1e3) / 1e9,
                 "speedup_vs_unfused_in_place": (inplace["ms_per_step"] / fms) if inplace else None,
                 "simulate": {"ms_per_step": sms, "gates_per_s": len(ops) / (sms / 1e3),
                              "moved_bytes_per_step": sbytes, "moved_gbs": sbytes / (sms / 1e3) / 1e9},
                 "norm": api.norm(c)}
        del c, fops

    # end to end through diaq_simulate: pinned host |j> in, pinned host result
    # out; its ops run in place with the identity-row skip, so the bytes are
    # the in-place bytes of each op
    e2e = None
    if not args.no_e2e:
        hin = torch.zeros(N, dtype=torch.complex128, pin_memory=True)
        hin[j] = 1.0
        hout = torch.empty(N, dtype=torch.complex128, pin_memory=True)
        w0 = torch.empty_like(a)
        ks = np.concatenate([np.arange(16), np.random.default_rng(7).integers(0, N, size=2048),
                             [N - 1]]).astype(np.int64)
        from_closed = np.exp(2j * np.pi * (((np.uint64(j) * ks.astype(np.uint64)) % np.uint64(N)).astype(np.float64)
                                           / N)) / math.sqrt(N)

        def e2e_run(sim_ops):
            api.simulate(sim_ops, hin, hout, w0)  # warm
            torch.cuda.synchronize()
            te = time.perf_counter()
            e_steps = max(1, min(args.steps, 3))
            legs = []
            for _ in range(e_steps):
                _, tl = api.simulate(sim_ops, hin, hout, w0, timeline=True)
                legs.append(tl)
            e_s = (time.perf_counter() - te) / e_steps
            # correctness: sampled amplitudes of the result against the closed form
            amp_err = float(np.max(np.abs(hout.numpy()[ks] - from_closed)))
            tl = [statistics.median(v[i] for v in legs) for i in range(3)]
            moved = api.simulate_bytes(sim_ops)  # merged diagonal runs and pairs counted as they run
            return {"value": world * len(ops) * bytes_op / e_s / 1e9, "unit": UNIT,
                    "h2d_bytes_per_step": N * 16, "d2h_bytes_per_step": N * 16, "ms_per_step": e_s * 1e3,
                    "gates_per_s": world * len(ops) / e_s, "ops": len(sim_ops),
                    "moved_gbs": world * moved / e_s / 1e9,
                    "timeline_ms": {"input_copied": tl[0], "last_op_done": tl[1], "output_copied": tl[2]},
                    "checked": {"sampled_amplitudes": int(len(ks)), "max_abs_err_vs_closed_form": amp_err,
                                "ok": bool(amp_err < 1e-12)}}

        # the circuit as a user runs it: each run of controlled phases fused
        # into one diagonal op (plan_fusion_diagonal), in place
        fops = api.build_fused(circ.gates, n, 6, 64, diagonal=True)
        e2e = e2e_run(fops)
        e2e["api"] = ("diaq_simulate on the qft-28 circuit with its runs of controlled phases fused into diagonal "
                      "ops (129 ops in place; pinned host buffers; the input copy overlaps the first op and the "
                      "output copy the last op, slice by slice)")
        e2e["accounting"] = ("value: the paper's algorithmic bytes of the circuit's 420 gates, 2 N s each, as in the "
                             "top-level value and the reference arm; moved_gbs: the bytes the in-place ops move")
        del fops
        e2e["unfused"] = e2e_run(ops)  # the same 420 ops as the timed step
        # the same copies alone, pinned host <-> device, 4 GiB each way
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c2 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        c0.record(stream)
        w0.copy_(hin, non_blocking=True)
        c1.record(stream)
        hout.copy_(w0, non_blocking=True)
        c2.record(stream)
        torch.cuda.synchronize()
        h2d_ms, d2h_ms = c0.elapsed_time(c1), c1.elapsed_time(c2)
        e2e["plain_pinned_copy"] = {"h2d_ms": h2d_ms, "d2h_ms": d2h_ms, "h2d_gbs": N * 16 / (h2d_ms / 1e3) / 1e9,
                                    "d2h_gbs": N * 16 / (d2h_ms / 1e3) / 1e9}
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
            # x, y and the stored values the SpMV reads (a gate op skips the
            # zeros stored where a diagonal crosses rows of another class);
            # the algorithmic count of the DiaQ SpMV is x, y and every stored
            # value, 2 N s + s sum_d (N - |d|)
            alg = op.apply_bytes()
            full = 2 * N * 16 + info["stored_bytes"]
            res[g.name] = {"apply_ms": ms, "gbs": alg / (ms / 1e3) / 1e9, "bytes": alg,
                           "gbs_all_stored_values": full / (ms / 1e3) / 1e9, "bytes_all_stored_values": full,
                           "stored_bytes": info["stored_bytes"], "build_ms": t_b0.elapsed_time(t_b1)}
            op.close()
        stored = {"ops": res, "accounting": "gbs: x, y and the stored values the SpMV reads; gbs_all_stored_values: "
                                            "x, y and every stored value, 2 N s + s sum_d (N - |d|)"}
        if not args.no_stored_step:
            # one whole step in the stored variant: each of the 420 ops is
            # materialised (Algorithm 2's diagonals, up to 12 GiB), applied
            # out of place and released before the next
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            x, y = a, b
            tot_alg = tot_full = 0
            marks = []
            for g in circ.gates:
                e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                e[0].record(stream)
                op = api.build(g, n, variant="stored")
                e[1].record(stream)
                api.apply(op, x, y)
                e[2].record(stream)
                marks.append(e)
                tot_alg += op.apply_bytes()
                tot_full += 2 * N * 16 + op.info()["stored_bytes"]
                op.close()
                x, y = y, x
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            mat_ms = sum(m[0].elapsed_time(m[1]) for m in marks)
            app_ms = sum(m[1].elapsed_time(m[2]) for m in marks)
            stored["step"] = {"workload": f"qft-{n} complex128, {len(circ.gates)} stored ops, each materialised, "
                                          "applied and released", "s_per_step": el, "gates_per_s": len(circ.gates) / el,
                              "materialise_ms": mat_ms, "apply_ms": app_ms,
                              "host_alloc_and_release_ms": el * 1e3 - mat_ms - app_ms,
                              "bytes_read_per_step": tot_alg, "bytes_all_stored_values_per_step": tot_full,
                              "apply_gbs": tot_alg / (app_ms / 1e3) / 1e9,
                              "apply_gbs_all_stored_values": tot_full / (app_ms / 1e3) / 1e9, "norm": api.norm(x)}

    shots = None
    if not args.no_sample:
        # the timed steps applied the QFT repeatedly; start again from |j>
        a.zero_()
        a[j] = 1.0
        x, y = a, b
        for op in ops:
            api.apply(op, x, y)
            x, y = y, x
        shots = bench_sample(api, a, n, j, stream)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128 (f64 arithmetic)", "data": "synthetic",
        "config": qft_config(n, len(ops), world),
        "gates_per_s": world * len(ops) * args.steps / (ms_total / 1e3),
        "apply_only_gbs": len(ops) * bytes_op / (apply_ms / 1e3) / 1e9,
        "per_class": per_class,
        "roofline": {"bound": "hbm", "kernel": "k_apply_small<double,2,1> (controlled phase, diagonal class)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": f"{peak_kind} hbm_gbs", "traffic": _traffic("cp_c128")},
        "e2e": e2e, "inplace": inplace, "fused": fused, "stored": stored, "sample": shots, "clocks": clocks,
        "gpu_launches": args.steps * (len(ops) + 2),
    }
    # free the QFT buffers before the secondary workloads
    del a, b, x0, ops
    torch.cuda.empty_cache()
    refs = {}
    if rank == 0 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(n, circ, j, budget_s=args.cpu_seconds)
        if not args.no_refs:
            refs = oracle_references(batch_count=args.batch_count)
            out["cpu_baseline_random"] = refs.pop("random_cpu")
    extras = {}
    if not args.no_adjoint:
        extras["adjoint"] = bench_adjoint(api, refs=refs.get("adjoint"))
    if not args.no_batch:
        extras["batch"] = bench_batch(api, count=args.batch_count, refs=refs.get("batch"))
    if not args.no_tfim:
        extras["tfim"] = bench_tfim(api, n=args.tfim_qubits, ref=refs.get("tfim"), ref_mag=refs.get("tfim_mag"))
    if not args.no_unitary:
        extras["unitary"] = bench_unitary(api)
    if not args.no_random:
        extras["random"] = bench_random(api, *REF_RANDOM, ref=refs.get("random"))
    if args.random_30:
        extras["random_30"] = bench_random_30(api, n=30)
    if extras:
        out["extras"] = extras
    return out


FP64_INSTR_PER_S = 0.528e12  # measured FP64 rate of GB300 (independent DFMA/DMUL/DADD chains)


def bench_sample(api, psi, n, j, stream, shots=1024, reps=10):
    """Born-rule shots (diaq_sample) of the QFT-28 state that the headline
    step leaves: 1024 shots per call (the paper's shots per run), complex128
    and a complex64 copy. The call reads the state once (the tile pass of
    the sum tree) and then descends the tree per shot. Bound: complex128 by
    the FP64 pipe (2 FMAs per amplitude), complex64 by HBM. Checked against
    the closed form: every |psi_k|^2 = 1/N, so shot u draws floor(u N) up to
    one index of rounding. read_gbs counts the state read once; the stored
    run and seg prefixes add 272 doubles per 4096 amplitudes (bytes_per_call)."""
    import torch
    N = 1 << n
    g = torch.Generator(device="cuda").manual_seed(0)
    u = torch.rand(shots, dtype=torch.float64, device="cuda", generator=g)
    out = {"workload": f"{shots} shots of the qft-{n} state per call", "shots": shots}
    hbm, _ = _peaks()
    for name, x, sz in (("c128", psi, 16), ("c64", None, 8)):
        if x is None:
            x = psi.to(torch.complex64)
        idx = torch.empty(shots, dtype=torch.int64, device="cuda")
        for _ in range(3):
            api.sample(x, u, idx)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            api.sample(x, u, idx)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        got = idx.cpu().numpy()
        ok = bool(np.all(np.abs(got - np.floor(u.cpu().numpy() * N)) <= 1))
        gbs = N * sz / (ms / 1e3) / 1e9
        rec = {"ms_per_call": ms, "shots_per_s": shots / (ms / 1e3), "read_gbs": gbs, "hbm_frac": gbs / hbm,
               "checked_closed_form": ok, "launches_per_call": 2 + (max(0, n - 12) + 7) // 8,
               "bytes_per_call": N * sz + (N // 4096) * 272 * 8}
        if name == "c128":
            floor_ms = 2 * N / FP64_INSTR_PER_S * 1e3
            rec.update({"bound": "fp64", "fp64_floor_ms": floor_ms, "fp64_frac": floor_ms / ms})
        else:
            rec["bound"] = "hbm"
        out[name] = rec
        del x
    return out


# FP64 instructions per amplitude of the complex128 sweep kernels, per gate
# kind: a Pauli rotation 4 forward (cos x + kappa x', a product and an FMA
# per part) and 10 reverse (U^dag on psi and lambda, and the 2-FMA gradient
# term); a fixed real gate (H) 4 forward, 8 reverse; CZ and other sign or
# permutation gates 0; a diagonal run (weight form) 4 forward, 11 reverse
# (2 for Im conj(l) p, 1 for W t, 8 for D^dag on both states); a chunk-form
# run of r rotations over c byte tables 4 (c - 1) + 4 forward and
# 4 (c - 1) + 2 + r + 8 reverse. The Pauli-sum lambda: 2 per term (the
# signed weights) and 4 per X-mask group, plus 2 for the energy. The reverse
# sweep stops at the earliest gate with a gradient term.
def fp64_per_amp(gates, obs, runs, chunks_run=None, scaled=False, product_layer_n=None):
    """(forward, reverse, lambda) FP64 instructions per amplitude of one
    energy + gradient of `gates`; with runs=True the diagonal runs are
    counted as the library forms them (chunks_run: (rotations, byte tables)
    of each chunk-form run in place of its member gates, or the weight form
    for runs of one-parameter rotations); with scaled=True rotations take
    the scaled form (one fused multiply-add per real component: 2 forward,
    2 + 2 + 2 reverse); with product_layer_n = n the leading fixed one-qubit
    gates on distinct qubits are written directly as a product state from
    per-byte tables (4 per further chunk of 8 qubits)."""
    def kind(g):
        if g.param >= 0:
            return "zrot" if set(g.gen) <= {"Z", "I"} else "rot"
        m = np.asarray(g.matrix)
        if np.count_nonzero(m - np.diag(np.diag(m))) == 0 and np.all(np.isin(np.diag(m), [1, -1])):
            return "sign"
        return "fixed"
    ks = [kind(g) for g in gates]
    first = next((i for i, k in enumerate(ks) if k in ("rot", "zrot")), len(ks))
    fwd = rev = 0
    layer = 0
    if product_layer_n:
        seen = set()
        while layer < len(gates) and not gates[layer].parametric and len(gates[layer].targets) == 1 \
                and gates[layer].targets[0] not in seen:
            seen.add(gates[layer].targets[0])
            layer += 1
        if layer:
            fwd += 4 * ((product_layer_n + 7) // 8 - 1)
    for i, k in enumerate(ks):
        if i < layer:
            continue
        if runs and k in ("zrot", "sign"):
            continue  # counted with the runs below
        rot_f, rot_r = (2, 6) if scaled else (4, 10)
        fwd += {"rot": rot_f, "zrot": rot_f, "fixed": 4, "sign": 0}[k]
        if i >= first:
            rev += {"rot": rot_r, "zrot": rot_r, "fixed": 8, "sign": 0}[k]
    if runs:
        for r_rot, c in (chunks_run or []):
            if c == 0:  # weight form
                fwd += 4
                rev += 11
            else:  # amplitudes by blocks of 256: the higher chunks' product once per block and lane
                ph = (4 if c > 1 else 0) + 4 * max(0, c - 2) / 8
                fwd += ph + 4
                # the term, its per-j and block sums, D^dag on psi and lambda; r_rot rotations on
                # bits fixed within a block but not for the thread take one signed addition per block
                rev += ph + 2 + 1 + 1 + 8 + r_rot / 8
    # lambda = H psi: per group of equal X masks the weight comes from a
    # table (no FP64 work when the coefficients are equal, else one complex
    # addition per further chunk of 8 terms), then 2 (real weight) or 4
    # multiply-adds; plus 2 for the energy
    grp = {}
    for x, z, c in zip(obs.xmask, obs.zmask, np.real(np.asarray(obs.coeff))):
        ny = bin(int(x) & int(z)).count("1") % 4
        kappa = complex(float(c)) * (1j ** ny)
        grp.setdefault(int(x), []).append(kappa)
    lam = 2
    for ks in grp.values():
        equal = all(k == ks[0] for k in ks)
        real = all(k.imag == 0 for k in ks)
        lam += (2 if real else 4) + (0 if equal else 2 * ((len(ks) + 7) // 8 - 1))
    return fwd, rev, lam


def bench_adjoint(api, n=20, layers=8, reps=3, refs=None):
    """Ansatz-20 energy + full gradient (320 parameters) by the adjoint sweep,
    complex128 and complex64, against the plain FP64 path: the
    parameter-shift gradient with one launch per gate (2 circuit
    evaluations per parameter, each 472 on-the-fly applies + the FP64
    expectation)."""
    import torch
    import synth
    circ = synth.ansatz(n=n, layers=layers, seed=0)
    obs = synth.ansatz_observable(n)
    out = {"workload": f"ansatz-{n}, {layers} layers, {circ.n_params} parameters, {len(circ.gates)} gates"}
    grads = {}
    energies_grads = {}
    for name, dt in (("c128", torch.complex128), ("c64", torch.complex64)):
        p0 = torch.zeros(1 << n, dtype=dt, device="cuda")
        p0[0] = 1
        wp, wl = torch.empty_like(p0), torch.empty_like(p0)
        for _ in range(2):
            e, g = api.adjoint_grad(circ.gates, circ.theta, obs.xmask, obs.zmask, obs.coeff, p0, wp, wl)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            e, g = api.adjoint_grad(circ.gates, circ.theta, obs.xmask, obs.zmask, obs.coeff, p0, wp, wl)
        el = (time.perf_counter() - t0) / reps
        grads[name] = g
        energies_grads[f"adjoint_{name}"] = (e, g)
        out[f"adjoint_{name}"] = {"grads_per_s": 1.0 / el, "ms_per_gradient": el * 1e3, "energy": e,
                                  "launches_per_gradient": 2 * len(circ.gates) + 4 + circ.n_params}
    # the same sweep recorded once as a CUDA graph and replayed per theta
    for name, dt in (("c128", torch.complex128), ("c64", torch.complex64)):
        plan = api.AdjointPlan(circ.gates, circ.n_params, (obs.xmask, obs.zmask, obs.coeff), n, dtype=dt)
        for _ in range(2):
            e, g = plan.run(circ.theta)
        t0 = time.perf_counter()
        r = 3 * reps
        for _ in range(r):
            e, g = plan.run(circ.theta)
        el = (time.perf_counter() - t0) / r
        out[f"adjoint_graph_{name}"] = {"grads_per_s": 1.0 / el, "ms_per_gradient": el * 1e3,
                                        "max_abs_grad_diff_vs_launch_path": float(np.max(np.abs(g - grads[name])))}
        # window-fused sweeps: blocks of <= w qubits, one launch per block, with
        # 1 or 4 threads per group, and the per-gate sweep at 1, 2 and 4
        # blocks per SM; the autotuner keeps the fastest
        tune = plan.autotune(circ.theta, reps=5)
        for _ in range(2):
            e, gw = plan.run(circ.theta)
        t0 = time.perf_counter()
        for _ in range(r):
            e, gw = plan.run(circ.theta)
        elw = (time.perf_counter() - t0) / r
        w, ln, nb = plan.sweep()
        energies_grads[f"adjoint_autotuned_{name}"] = (e, gw)
        out[f"adjoint_autotuned_{name}"] = {
            "window": w, "lanes": ln, "blocks": plan.blocks(), "launches_per_sweep": nb, "grads_per_s": 1.0 / elw,
            "ms_per_gradient": elw * 1e3, "max_abs_grad_diff_vs_launch_path": float(np.max(np.abs(gw - grads[name]))),
            "device_ms_by_sweep": {f"w{tw}_l{tl}" + (f"_b{tb}" if tw == 0 else ""): m
                                   for tw, tl, tb, m in tune["tried"]}}
        plan.close()
    out["c64_vs_c128_max_abs_grad_diff"] = float(np.max(np.abs(grads["c64"] - grads["c128"])))
    # the same plan, complex128: gate by gate (diagonal runs off), and with
    # the rotations unscaled
    def timed_plan(runs, scaled, pairs=True):
        plan = api.AdjointPlan(circ.gates, circ.n_params, (obs.xmask, obs.zmask, obs.coeff), n,
                               dtype=torch.complex128)
        plan.set_runs(runs)
        plan.set_scaled(scaled)
        plan.set_pairs(pairs)
        info = plan.runs(), plan.scaled()
        for _ in range(2):
            plan.run(circ.theta)
        t0 = time.perf_counter()
        for _ in range(3 * reps):
            plan.run(circ.theta)
        el = (time.perf_counter() - t0) / (3 * reps)
        plan.close()
        return el, info

    el_off, _ = timed_plan(False, True)
    out["adjoint_gate_by_gate_graph_c128"] = {"ms_per_gradient": el_off * 1e3, "grads_per_s": 1.0 / el_off}
    el_us, ((on, n_runs, steps), _) = timed_plan(True, False)
    out["adjoint_unscaled_graph_c128"] = {"ms_per_gradient": el_us * 1e3, "grads_per_s": 1.0 / el_us}
    el_np, _ = timed_plan(True, True, pairs=False)
    out["adjoint_unpaired_graph_c128"] = {"ms_per_gradient": el_np * 1e3, "grads_per_s": 1.0 / el_np,
                                          "note": "one launch per rotation (fused rotation pairs off)"}
    # FP64 floor of a complex128 gradient (FP64-bound: the 16 MiB states stay in L2)
    N = 1 << n
    chunks = (n + 7) // 8
    # the reverse chunk-form kernel takes a per-block term only for rotations
    # on bits at or above 11 + the trailing zeros of its block count
    # (blocks = min(N / 512, 2 SMs), 256 threads each)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks = min(N // 512, 2 * sms)
    fixed_bits = 11 + (blocks & -blocks).bit_length() - 1
    varying = max(0, n - fixed_bits)
    best = out["adjoint_autotuned_c128"]["ms_per_gradient"]
    scaled_best = out["adjoint_autotuned_c128"]["window"] == 0
    f0, r0, l0 = fp64_per_amp(circ.gates, obs, runs=False)
    fu, ru, lu = fp64_per_amp(circ.gates, obs, runs=True, chunks_run=[(varying, chunks)] * layers)
    f1, r1, l1 = fp64_per_amp(circ.gates, obs, runs=True, chunks_run=[(varying, chunks)] * layers,
                              scaled=scaled_best)
    out["roofline_c128"] = {
        "bound": "fp64", "unit": "FP64 instructions", "peak_instr_per_s": FP64_INSTR_PER_S,
        "peak_source": "measured FP64 probe (independent DFMA chains), not MEASURED_PEAKS.json",
        "diagonal_runs": n_runs, "launches_per_direction": steps, "scaled_rotations": scaled_best,
        "fp64_instr_per_gradient": (f1 + r1 + l1) * N, "floor_ms": (f1 + r1 + l1) * N / FP64_INSTR_PER_S * 1e3,
        "achieved_ms": best, "frac": (f1 + r1 + l1) * N / FP64_INSTR_PER_S * 1e3 / best,
        "unscaled_fp64_instr_per_gradient": (fu + ru + lu) * N,
        "unscaled_floor_ms": (fu + ru + lu) * N / FP64_INSTR_PER_S * 1e3,
        "frac_of_unscaled_floor": (fu + ru + lu) * N / FP64_INSTR_PER_S * 1e3 / best,
        "gate_by_gate_fp64_instr_per_gradient": (f0 + r0 + l0) * N,
        "gate_by_gate_floor_ms": (f0 + r0 + l0) * N / FP64_INSTR_PER_S * 1e3,
        "frac_of_gate_by_gate_floor": (f0 + r0 + l0) * N / FP64_INSTR_PER_S * 1e3 / best,
        "bytes_per_gradient": N * 16 * (2 * steps + 4 * steps + 2),
        "note": "per amplitude: rotation 2 forward / 6 reverse scaled (4 / 10 unscaled); chunk-form diagonal run "
                "(RZ layer + CZ ladder) p + 4 forward, p + 12 + v / 8 reverse, p = 4 + 4 (c - 2) / 8 for the phase "
                "(amplitudes by blocks of 256, the higher chunks once per block; v rotations on bits at or above 11 + "
                "the block count's trailing zeros); lambda 2 per real term group (weights from tables) + 2 for the "
                "energy"}
    for name in ("c128", "c64"):
        # what the graph plan and the window-fused sweep add over the
        # one-launch-per-gate adjoint sweep (the same algorithm)
        out[f"speedup_graph_vs_launch_adjoint_{name}"] = (out[f"adjoint_graph_{name}"]["grads_per_s"]
                                                         / out[f"adjoint_{name}"]["grads_per_s"])
        out[f"speedup_autotuned_vs_launch_adjoint_{name}"] = (out[f"adjoint_autotuned_{name}"]["grads_per_s"]
                                                             / out[f"adjoint_{name}"]["grads_per_s"])
    if refs is not None:
        p = refs["params"]
        out["vs_oracle"] = {"reference": f"FP64 oracle energy and parameter-shift gradient at {len(p)} sampled "
                                         "parameters (cpu_baseline leg)"}
        for key in ("adjoint_c128", "adjoint_c64", "adjoint_autotuned_c128", "adjoint_autotuned_c64"):
            e, g = energies_grads[key]
            out["vs_oracle"][key] = {"energy_abs_err": abs(e - refs["energy"]),
                                     "grad_max_abs_err": float(np.max(np.abs(g[p] - refs["grad"])))}
    # plain FP64 path: one circuit evaluation = 472 applies + expectation
    ops = [api.build(g, n, theta=circ.theta) for g in circ.gates]
    x = torch.zeros(1 << n, dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)

    def evaluate():
        a, b = x, y
        a.zero_()
        a[0] = 1
        for op in ops:
            api.apply(op, a, b)
            a, b = b, a
        return api.expect(a, obs.xmask, obs.zmask, obs.coeff).real

    evaluate()
    t0 = time.perf_counter()
    k = 6
    for _ in range(k):
        evaluate()
    t_eval = (time.perf_counter() - t0) / k
    n_eval = 2 * circ.n_params
    out["plain_fp64_param_shift"] = {"ms_per_evaluation": t_eval * 1e3, "evaluations_per_gradient": n_eval,
                                     "grads_per_s": 1.0 / (n_eval * t_eval),
                                     "note": f"timed on {k} evaluations, a gradient needs {n_eval}"}
    out["speedup_adjoint_c128_vs_plain"] = out["adjoint_c128"]["grads_per_s"] / out["plain_fp64_param_shift"]["grads_per_s"]
    out["speedup_adjoint_c64_vs_plain"] = out["adjoint_c64"]["grads_per_s"] / out["plain_fp64_param_shift"]["grads_per_s"]
    for name in ("c128", "c64"):
        out[f"speedup_adjoint_graph_{name}_vs_plain"] = (out[f"adjoint_graph_{name}"]["grads_per_s"]
                                                        / out["plain_fp64_param_shift"]["grads_per_s"])
        out[f"speedup_adjoint_autotuned_{name}_vs_plain"] = (out[f"adjoint_autotuned_{name}"]["grads_per_s"]
                                                            / out["plain_fp64_param_shift"]["grads_per_s"])
    return out


def bench_batch(api, count=256, reps=3, plain=True, shape=None, dtypes=("c64", "c128"), refs=None):
    """QAOA MaxCut batch: `count` circuits on random 3-regular graphs,
    n in {14..22}, p = 4: energy + 8-parameter gradient per circuit in one
    persistent launch replayed from a CUDA graph (launch shape chosen by the
    autotuner on a 16-circuit proxy batch of the same size mix), complex64
    and complex128, against the plain path: diaq_adjoint_grad per circuit in
    FP64 (one launch per gate)."""
    import torch
    import synth
    inst = synth.qaoa_batch(count, seed=0)
    theta = np.concatenate([c.theta for c, _ in inst])
    desc = [(c.n, c.gates, c.n_params, (o.xmask, o.zmask, o.coeff)) for c, o in inst]
    sizes = sorted(set(c.n for c, _ in inst))
    out = {"workload": f"qaoa batch: {count} circuits, n in {sizes}, p=4, energy + 8 grads each"}
    energies = {}
    for name, dt in (("c64", torch.complex64), ("c128", torch.complex128)):
        if name not in dtypes:
            continue
        if shape is None:
            proxy = api.Batch(desc[:16], dtype=dt)
            tune = proxy.autotune(np.concatenate([c.theta for c, _ in inst[:16]]), reps=1)
            proxy.close()
        else:
            tune = {"best_cluster": shape[0], "best_threads": shape[1], "best_window": shape[2] if len(shape) > 2 else 0,
                    "best_lanes": shape[3] if len(shape) > 3 else 1, "best_ms": None, "tried": []}
        b = api.Batch(desc, dtype=dt)
        b.set_sweep(tune.get("best_window", 0), tune.get("best_lanes", 1))
        b.set_launch(tune["best_cluster"], tune["best_threads"])
        E, G = b.run(theta)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            E, G = b.run(theta)
        el = (time.perf_counter() - t0) / reps
        energies[name] = E
        if refs:
            out.setdefault("vs_oracle", {"reference": f"FP64 oracle energies and parameter-shift gradients of "
                                                      f"{len(refs)} 14-qubit instances (cpu_baseline leg)",
                                         "instances": sorted(int(i) for i in refs)})
            out["vs_oracle"][name] = {
                "energy_max_abs_err": max(abs(E[i] - refs[i][0]) for i in refs),
                "grad_max_abs_err": max(float(np.max(np.abs(G[i] - refs[i][1]))) for i in refs)}
        q = b.query()
        unscaled_ms = None
        if b.scaled()[1]:  # the same batch with the rotations unscaled
            b.set_scaled(False)
            b.run(theta)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                b.run(theta)
            unscaled_ms = (time.perf_counter() - t0) / reps * 1e3
            b.set_scaled(True)
        out[f"batched_{name}"] = {"circuits_per_s": count / el, "ms_per_batch": el * 1e3,
                                  "scaled": b.scaled()[1], "unscaled_ms_per_batch": unscaled_ms,
                                  "diagonal_runs": b.runs()[1],
                                  "cluster": q["cluster"], "threads": q["threads"], "window": b.sweep()[0],
                                  "lanes": b.sweep()[1],
                                  "teams": q["teams"],
                                  "arena_bytes": q["arena_bytes"], "launches_per_batch": 2,
                                  "tuning": {"proxy_best_ms": tune["best_ms"], "shapes_tried": len(tune["tried"])}}
        b.close()
    if len(energies) == 2:
        out["c64_vs_c128_max_abs_energy_diff"] = float(np.max(np.abs(energies["c64"] - energies["c128"])))
    if plain and "c128" in energies:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e_plain = []
        for c, o in inst:
            p0 = torch.zeros(1 << c.n, dtype=torch.complex128, device="cuda")
            p0[0] = 1
            e, g = api.adjoint_grad(c.gates, c.theta, o.xmask, o.zmask, o.coeff, p0, torch.empty_like(p0),
                                    torch.empty_like(p0))
            e_plain.append(e)
        el = time.perf_counter() - t0
        out["plain_fp64_per_circuit"] = {"circuits_per_s": count / el, "ms_per_batch": el * 1e3}
        # FP64 floor of the complex128 batch (sum over circuits of N x
        # instructions per amplitude, gate by gate and with the cost layers
        # as weight-form diagonal runs)
        scaled_best = out["batched_c128"]["scaled"]
        fl0 = flu = fl1 = 0.0
        for c, o in inst:
            f0, r0, l0 = fp64_per_amp(c.gates, o, runs=False)
            fu, ru, lu = fp64_per_amp(c.gates, o, runs=True, chunks_run=[(0, 0)] * 4)
            f1, r1, l1 = fp64_per_amp(c.gates, o, runs=True, chunks_run=[(0, 0)] * 4, scaled=scaled_best,
                                      product_layer_n=c.n)
            fl0 += (1 << c.n) * (f0 + r0 + l0)
            flu += (1 << c.n) * (fu + ru + lu)
            fl1 += (1 << c.n) * (f1 + r1 + l1)
        bt = out["batched_c128"]["ms_per_batch"]
        out["roofline_c128"] = {
            "bound": "fp64", "unit": "FP64 instructions", "peak_instr_per_s": FP64_INSTR_PER_S,
            "peak_source": "measured FP64 probe (independent DFMA chains), not MEASURED_PEAKS.json",
            "scaled_rotations": scaled_best,
            "fp64_instr_per_batch": fl1, "floor_ms": fl1 / FP64_INSTR_PER_S * 1e3, "achieved_ms": bt,
            "frac": fl1 / FP64_INSTR_PER_S * 1e3 / bt,
            "unscaled_fp64_instr_per_batch": flu, "unscaled_floor_ms": flu / FP64_INSTR_PER_S * 1e3,
            "frac_of_unscaled_floor": flu / FP64_INSTR_PER_S * 1e3 / bt,
            "gate_by_gate_fp64_instr_per_batch": fl0,
            "gate_by_gate_floor_ms": fl0 / FP64_INSTR_PER_S * 1e3,
            "frac_of_gate_by_gate_floor": fl0 / FP64_INSTR_PER_S * 1e3 / bt}
        out["batched_c128_vs_plain_max_abs_energy_diff"] = float(np.max(np.abs(np.array(e_plain) - energies["c128"])))
        out["speedup_batched_c128_vs_plain"] = out["batched_c128"]["circuits_per_s"] / out["plain_fp64_per_circuit"]["circuits_per_s"]
        out["speedup_batched_c64_vs_plain"] = out["batched_c64"]["circuits_per_s"] / out["plain_fp64_per_circuit"]["circuits_per_s"]
    return out


def bench_tfim(api, n=28, steps=10, dt=0.1, J=1.0, h=0.7, ref=None, ref_mag=None):
    """Trotterised 1D transverse-field Ising model (the paper's
    Hamiltonian-simulation workload): `steps` first-order Trotter steps of
    ZZ bond rotations and X field rotations, in place, complex128 and
    complex64, read out as the average magnetisation (FP64 reduction)."""
    import torch
    import synth
    circ = synth.tfim(n, steps, dt, J=J, h=h)
    obs = synth.magnetisation_observable(n)
    N = 1 << n
    out = {"workload": f"tfim-{n}, {steps} Trotter steps (dt {dt}, J {J}, h {h}): {len(circ.gates)} gates, "
                       "in place + magnetisation"}
    stream = torch.cuda.current_stream()
    mags = {}
    for name, dt_ in (("c128", torch.complex128), ("c64", torch.complex64)):
        ops = [api.build(g, n, dtype=dt_, theta=circ.theta) for g in circ.gates]
        nbytes = sum(op.apply_bytes(in_place=True) for op in ops)
        x = torch.zeros(N, dtype=dt_, device="cuda")
        for rep in range(2):  # the first pass warms up, the second is timed
            x.zero_()
            x[0] = 1
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for op in ops:
                api.apply(op, x, x)
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        mags[name] = api.expect(x, obs.xmask, obs.zmask, obs.coeff).real
        out[name] = {"ms_per_circuit": ms, "gates_per_s": len(ops) / (ms / 1e3), "gbs": nbytes / (ms / 1e3) / 1e9,
                     "magnetisation": mags[name], "norm": api.norm(x)}
        del ops
        # the same circuit as a user runs it: each run of bond rotations fused
        # into diagonal ops of up to 6 qubits (plan_fusion_diagonal), field
        # rotations single, all through diaq_simulate in place on the device
        # state (complex128 field rotations take its scaled form)
        fops = api.build_fused(circ.gates, n, 6, 64, dtype=dt_, theta=circ.theta, diagonal=True)
        fbytes = api.simulate_bytes(fops)
        for rep in range(2):
            x.zero_()
            x[0] = 1
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            f0.record(stream)
            api.simulate(fops, x, x, x)
            f1.record(stream)
            torch.cuda.synchronize()
        fms = f0.elapsed_time(f1)
        fmag = api.expect(x, obs.xmask, obs.zmask, obs.coeff).real
        out[name + "_fused"] = {"ops": len(fops), "ms_per_circuit": fms, "gates_per_s": len(circ.gates) / (fms / 1e3),
                                "moved_gbs": fbytes / (fms / 1e3) / 1e9, "speedup_vs_unfused": ms / fms,
                                "magnetisation_abs_diff_vs_unfused": abs(fmag - mags[name])}
        del fops, x
    out["c64_vs_c128_magnetisation_diff"] = abs(mags["c64"] - mags["c128"])
    if ref is not None:
        # the same Trotter circuit at REF_TFIM qubits against the FP64 oracle
        m = REF_TFIM
        cc = synth.tfim(m, steps, dt, J=J, h=h)
        ob = synth.magnetisation_observable(m)
        chk = {"qubits": m, "reference": "FP64 oracle (cpu_baseline leg)"}
        for name, dt_ in (("c128", torch.complex128), ("c64", torch.complex64)):
            ops = [api.build(g, m, dtype=dt_, theta=cc.theta) for g in cc.gates]
            x = torch.zeros(1 << m, dtype=dt_, device="cuda")
            x[0] = 1
            for op in ops:
                api.apply(op, x, x)
            rec = state_errors(x.cpu().numpy(), ref)
            rec["magnetisation_abs_err_vs_oracle"] = abs(api.expect(x, ob.xmask, ob.zmask, ob.coeff).real - ref_mag)
            chk[name] = rec
            del ops, x
        out["check_vs_oracle"] = chk
    return out


def bench_unitary(api):
    """Unitary simulation by chained device DiaQ products (Algorithm 1), with
    all-zero diagonals pruned after each product: GHZ-12 (stays sparse) and
    TFIM-10 with 2 Trotter steps (fills in), complex128. Reports the time per
    chain, the diagonals and non-zeros at the end, and the peak."""
    import torch
    import synth
    out = {}
    for name, n, circ in (("ghz", 12, synth.ghz(12)), ("tfim", 10, synth.tfim(10, 2, 0.1, J=1.0, h=0.7))):
        N = 1 << n
        op, nd, nz = api.unitary_chain(circ.gates, n, theta=circ.theta if circ.n_params else None)
        del op
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        op, nd, nz = api.unitary_chain(circ.gates, n, theta=circ.theta if circ.n_params else None)
        el = time.perf_counter() - t0
        out[f"{name}-{n}"] = {"gates": len(circ.gates), "ms_per_chain": el * 1e3,
                               "products_per_s": (len(circ.gates) - 1) / el,
                               "final_diagonals": int(nd[-1]), "final_nnz": int(nz[-1]),
                               "final_sparsity": 1.0 - float(nz[-1]) / (N * N),
                               "min_sparsity": 1.0 - float(np.max(nz)) / (N * N),
                               "max_diagonals": int(np.max(nd))}
        del op
    return out


def _c64_bound(ks) -> float:
    """Worst-case 2-norm error bound of a complex64 circuit of unitary gates
    on k_i qubits (k = 0 for gates whose entries are 0 or +-1, applied
    exactly): per gate ((2^(k+1) + 1) 1.01 + sqrt 2) 2^(k/2) units of 2^-24,
    summed over the gates (each later gate is unitary)."""
    u = 2.0 ** -24
    return 1.01 * u * sum(((2 ** (k + 1) + 1) * 1.01 + math.sqrt(2.0)) * 2.0 ** (k / 2.0) for k in ks if k > 0)


def bench_random(api, n=24, depth=40, ref=None):
    """Random layered circuit (Haar U(2) on every qubit + CZ on a random
    matching per layer) at the largest size the oracle runs in seconds: one
    in-place pass in complex64 and complex128, plain and with
    commutation-aware fusion (max K 3, depth 6), each with its fidelity and
    max amplitude error against the FP64 oracle's state (and, for
    complex64, the worst-case rounding bound). The state (128 or 256 MiB)
    is about the size of L2, so the times here are not an HBM figure; the
    30-qubit line gives that."""
    import torch
    import synth
    circ = synth.random_layered(n, depth, seed=0)
    N = 1 << n
    out = {"workload": f"random-{n} depth {depth}: {len(circ.gates)} gates, in place",
           "reference": "FP64 oracle (cpu_baseline leg)" if ref is not None else None}
    for name, dt in (("c64", torch.complex64), ("c128", torch.complex128)):
        for mode in ("plain", "fused", "simulate"):
            if mode == "fused":
                ops = api.build_fused(circ.gates, n, 3, 6, dtype=dt, commuting=True)
                ks = [op.info()["k"] for op in ops]
            else:
                ops = [api.build(g, n, dtype=dt) for g in circ.gates]
                ks = [0 if g.name == "cz" else g.k for g in circ.gates]
            x = torch.zeros(N, dtype=dt, device="cuda")
            for rep in range(2):  # the first pass warms up
                x.zero_()
                x[0] = 1
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                if mode == "simulate":  # the user-level call: pairs and merged CZ runs
                    api.simulate(ops, x, x, x)
                else:
                    for op in ops:
                        api.apply(op, x, x)
                torch.cuda.synchronize()
                el = time.perf_counter() - t0
            key = name + ("" if mode == "plain" else "_" + mode)
            rec = {"ops": len(ops), "s_per_circuit": el, "gates_per_s": len(circ.gates) / el, "norm": api.norm(x)}
            if ref is not None:
                rec.update(state_errors(x.cpu().numpy(), ref))
            if name == "c64":
                b = _c64_bound(ks)
                rec["max_abs_err_bound"] = b
                rec["infidelity_bound"] = b * b / (1.0 - b) ** 2
            out[key] = rec
            del ops, x
    return out


def bench_random_30(api, n=30, depth=40):
    """Random layered circuit at 30 qubits (8 or 16 GiB state), complex64
    vs complex128, one pass each; fusion depth chosen by the autotuner for
    complex64. The oracle does not run at this size, so the complex64 state
    is compared with the complex128 GPU state, which matches the oracle to
    1e-12 wherever the oracle runs (24 qubits in the random line)."""
    import torch
    import synth
    circ = synth.random_layered(n, depth, seed=0)
    N = 1 << n
    out = {"workload": f"random-{n} depth {depth}: {len(circ.gates)} gates",
           "reference": "complex128 GPU state (oracle-pinned at <= 24 qubits)"}
    res = {}
    for name, dt, s in (("c64", torch.complex64, 8), ("c128", torch.complex128, 16)):
        ops = [api.build(g, n, dtype=dt) for g in circ.gates]
        # in place: CZ gates take the identity-row skip, so count the bytes moved
        moved = sum(op.apply_bytes(in_place=True) for op in ops)
        x = torch.zeros(N, dtype=dt, device="cuda")
        x[0] = 1
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for op in ops:
            api.apply(op, x, x)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        res[name] = x
        out[name] = {"s_per_circuit": el, "gates_per_s": len(ops) / el, "gbs": moved / el / 1e9,
                     "bytes_moved": moved, "norm": api.norm(x)}
        del ops
    a = res["c128"]
    b = res["c64"].to(torch.complex128)
    ov = torch.vdot(a, b)
    out["c64_fidelity_vs_c128"] = float((ov.abs() ** 2 / (torch.vdot(a, a).real * torch.vdot(b, b).real)).item())
    out["c64_max_abs_err_vs_c128"] = float((a - b).abs().max().item())
    del b
    res.pop("c64")
    w = torch.zeros(N, dtype=torch.complex64, device="cuda")
    w[0] = 1
    prefix = circ.gates[: 5 * (n + n // 2)]
    tunes = {}
    for mk in (2, 3):
        tunes[mk] = api.autotune_fusion(prefix, n, w, max_k=mk, max_depth=8, commuting=True)
    mk = min(tunes, key=lambda m: min(tunes[m]["ms"]))
    d = tunes[mk]["best_depth"]
    ops = api.build_fused(circ.gates, n, mk, d, dtype=torch.complex64, commuting=True)
    w.zero_()
    w[0] = 1
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for op in ops:
        api.apply(op, w, w)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    out["c64_fused"] = {"max_k": mk, "depth": d, "ops": len(ops), "s_per_circuit": el,
                        "gates_per_s": len(circ.gates) / el,
                        "tuning_ms_by_depth": {str(m): t["ms"] for m, t in tunes.items()}}
    wf = w.to(torch.complex128)
    out["c64_fused"]["fidelity_vs_c128"] = float(
        (torch.vdot(a, wf).abs() ** 2 / (torch.vdot(a, a).real * torch.vdot(wf, wf).real)).item())
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


# Sizes of the oracle reference runs behind the precision fields of the
# secondary workloads (each a few seconds to ~20 s on the host cores).
REF_RANDOM = (24, 40)      # random layered: qubits, depth
REF_TFIM = 22              # TFIM qubits (10 Trotter steps, as the timed line)
REF_ADJOINT_PARAMS = 8     # Ansatz-20 parameters checked by parameter shift
REF_BATCH_INSTANCES = 4    # 14-qubit QAOA instances of the batch checked


def oracle_references(batch_count=256):
    """Part of the cpu_baseline leg (rank 0, outside every timed region):
    the FP64 oracle's results that the secondary workloads' GPU results are
    compared with (fidelity and max amplitude error of final states; energy
    and sampled gradient entries). Also times the oracle on the random
    layered circuit."""
    import oracle
    import synth
    refs = {}
    n, depth = REF_RANDOM
    circ = synth.random_layered(n, depth, seed=0)
    t0 = time.perf_counter()
    refs["random"] = oracle.run_circuit(circ, synth.basis_state(n, 0))
    el = time.perf_counter() - t0
    refs["random_cpu"] = {"gates_per_s": len(circ.gates) / el, "s_per_circuit": el, "cores": oracle.threads(),
                          "kind": "oracle", "sample": f"random-{n} depth {depth}, whole circuit, complex128"}
    tc = synth.tfim(REF_TFIM, 10, 0.1, J=1.0, h=0.7)
    refs["tfim"] = oracle.run_circuit(tc, synth.basis_state(REF_TFIM, 0), tc.theta)
    refs["tfim_mag"] = oracle.expect(refs["tfim"], synth.magnetisation_observable(REF_TFIM)).real
    ac = synth.ansatz(n=20, layers=8, seed=0)
    ao = synth.ansatz_observable(20)
    a0 = synth.basis_state(20, 0)
    params = np.linspace(0, ac.n_params - 1, REF_ADJOINT_PARAMS).astype(int)
    refs["adjoint"] = {"energy": oracle.energy(ac, ao, a0), "params": params,
                       "grad": oracle.param_shift_grad(ac, ao, a0, params=params)[params]}
    inst = synth.qaoa_batch(batch_count, seed=0)
    picked = [i for i, (c, _) in enumerate(inst) if c.n == 14][:REF_BATCH_INSTANCES]
    refs["batch"] = {}
    for i in picked:
        c, o = inst[i]
        p0 = synth.basis_state(c.n, 0)
        refs["batch"][i] = (oracle.energy(c, o, p0), oracle.param_shift_grad(c, o, p0))
    return refs


def state_errors(got, want) -> dict:
    """Fidelity |<a|b>|^2 / (<a|a><b|b>) and max amplitude error of a GPU
    state against the oracle's (numpy on the host copies)."""
    a = np.asarray(want, dtype=np.complex128)
    b = np.asarray(got, dtype=np.complex128)
    f = abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real)
    return {"fidelity_vs_oracle": float(f), "infidelity_vs_oracle": float(1.0 - f),
            "max_abs_err_vs_oracle": float(np.max(np.abs(a - b)))}


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
        "config": qft_config(n, len(circ.gates), world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                         "sample": f"{per_step} of the {len(circ.gates)} qft-{n} ops per step, FP64 oracle"},
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
    ap.add_argument("--no-stored-step", action="store_true")
    ap.add_argument("--no-sample", action="store_true")
    ap.add_argument("--no-fused", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-inplace", action="store_true")
    ap.add_argument("--no-tfim", action="store_true")
    ap.add_argument("--no-unitary", action="store_true")
    ap.add_argument("--tfim-qubits", type=int, default=28)
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--batch-only", action="store_true", help="profiling entry: one batch run, fixed shape")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="profiling entry: replays of the ansatz-20 adjoint plan at a fixed sweep")
    ap.add_argument("--adjoint-dtype", default="c128", choices=["c64", "c128"])
    ap.add_argument("--adjoint-window", type=int, default=0)
    ap.add_argument("--adjoint-lanes", type=int, default=1)
    ap.add_argument("--adjoint-reps", type=int, default=3)
    ap.add_argument("--adjoint-blocks", type=int, default=0, help="per-gate sweep blocks (0: two per SM)")
    ap.add_argument("--adjoint-qubits", type=int, default=20)
    ap.add_argument("--batch-cluster", type=int, default=8)
    ap.add_argument("--batch-threads", type=int, default=256)
    ap.add_argument("--batch-dtype", default="c64", choices=["c64", "c128"])
    ap.add_argument("--batch-window", type=int, default=0)
    ap.add_argument("--batch-lanes", type=int, default=1)
    ap.add_argument("--no-random", action="store_true", help="skip the random layered circuit at 24 qubits")
    ap.add_argument("--random-30", action="store_true", help="also run the random layered circuit at 30 qubits")
    ap.add_argument("--no-refs", action="store_true", help="skip the oracle reference runs of the precision fields")
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    launched = int(os.environ.get("WORLD_SIZE", "1"))
    if args.gpus != launched:
        # one process per GPU: N GPUs need N ranks (torchrun --nproc-per-node N)
        print(f"bench.py --gpus {args.gpus} needs {args.gpus} ranks, but WORLD_SIZE is {launched}: launch it as "
              f"python -m torch.distributed.run --nproc-per-node {args.gpus} bench.py --gpus {args.gpus} ...",
              file=sys.stderr)
        sys.exit(2)
    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        world = int(os.environ.get("WORLD_SIZE", "1"))
        if rank != 0:
            return
        print(json.dumps(run_reference(args, rank, world)), flush=True)
        return
    if args.batch_only:
        # profiling entry: one batch at a fixed team shape, no autotuning
        import torch  # noqa: F401
        from paper_2405_01250_gb300 import build as B
        B.build()
        from paper_2405_01250_gb300 import api
        print(json.dumps(bench_batch(api, count=args.batch_count, reps=1, plain=False,
                                     shape=(args.batch_cluster, args.batch_threads, args.batch_window,
                                            args.batch_lanes),
                                     dtypes=(args.batch_dtype,))), flush=True)
        return
    if args.adjoint_only:
        # profiling entry: the plan at a fixed sweep, 2 warm-up replays and
        # adjoint_reps timed ones (host clock), no autotuning
        import torch
        import synth
        from paper_2405_01250_gb300 import build as B
        B.build()
        from paper_2405_01250_gb300 import api
        nq = args.adjoint_qubits
        circ = synth.ansatz(n=nq, layers=8, seed=0)
        obs = synth.ansatz_observable(nq)
        dt = torch.complex128 if args.adjoint_dtype == "c128" else torch.complex64
        plan = api.AdjointPlan(circ.gates, circ.n_params, (obs.xmask, obs.zmask, obs.coeff), nq, dtype=dt)
        plan.set_sweep(args.adjoint_window, args.adjoint_lanes)
        plan.set_blocks(args.adjoint_blocks)
        for _ in range(2):
            plan.run(circ.theta)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.adjoint_reps):
            e, _ = plan.run(circ.theta)
        el = (time.perf_counter() - t0) / max(1, args.adjoint_reps)
        print(json.dumps({"workload": f"ansatz-{nq} adjoint plan", "dtype": args.adjoint_dtype, "sweep": plan.sweep(),
                          "runs": plan.runs(), "scaled": plan.scaled(), "pairs": plan.pairs(),
                          "blocks": plan.blocks(), "ms_per_gradient": el * 1e3, "energy": e}), flush=True)
        plan.close()
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
