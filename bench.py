#!/usr/bin/env python
"""Throughput benchmark of the GB300 Lomb-Scargle path.

A step is one pass of the whole path over one batch resident in HBM: the
prologue (centring, phase records), the work-queue order, the persistent
trig-sum kernel with its fused power/argmax/top-3 epilogue and the finalize
kernel, replayed as one CUDA graph (``lsp_plan_execute``) with the autotuned
configuration.  The default workload is the largest batch: 100000 objects,
N_t log-uniform in [10, 2000] with a seasonal cadence, N_f = 50000 on
[0.24, 12) c/d, FP32 sums with FP64/fixed-point phases, argmax and top-3.

One JSON line is printed by rank 0.  ``value`` is objects/s over all ranks;
``e2e`` is the same metric through the host-buffer entry point with the
copies inside the timed region; ``roofline`` relates the main kernel's
measured pair rate to the FP32-pipe bound; ``cpu_baseline`` times the FP64
CPU oracle on a bounded sample of the same workload on this host's cores;
``learned`` (default workload, one GPU) times the learned proposal path
(``lsp_propose_refine``, one call) against the plain full grid on 100000
survey-shaped objects with N_f = 1e5, with its recovery of the full grid's
periods.  Under torchrun the batch is sharded over the ranks by N_t
(``shard.shard_ranges``; strong scaling) and the peaks are gathered on rank 0
(``shard.gather_peaks``); ``--replicas`` gives every rank its own batch
instead (weak scaling).

``--impl reference`` times the oracle alone (the CPU reference arm).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "objects/sec and trig-sum evals/s (N_t*N_f) vs FP32 roofline; learned vs plain"
OPS_PER_PAIR = 8           # roofline work unit: one pair in the rotation-recurrence form costs 2 FMUL +
                           # 2 FFMA (rotation) + 4 FFMA (XC, XS, CC, CS) on the FP32 pipe
KERNEL_OPS_PER_PAIR = 6    # what the kernels spend: a chain of K pairs takes one rotation (4) and K - 2
                           # three-term steps (2 each), 2K in all, plus the 4 FFMA of the sums
FP32_LANES_PER_SM = 128    # FP32 lanes per SM per clock
FP64_LANES_PER_SM = 2      # FP64 FMAs per SM per clock: 1.25 TFLOP/s nominal / (2 x 152 SMs x 2.07 GHz)

WORKLOADS = {
    "ragged_survey": dict(kind="batch", top_k=1, power=False, cpu_sample=64, ref_per_step=6,
                          desc="10000 objects, N_t~U{50..500}, seasonal cadence, N_f=1e5 on [0.24,12) c/d, argmax only"),
    "ragged_lognormal": dict(kind="batch", top_k=3, power=False, cpu_sample=48, ref_per_step=6,
                             desc="100000 objects, N_t log-uniform in [10,2000], N_f=5e4 on [0.24,12) c/d, argmax + top-3"),
    "single_small": dict(kind="single", top_k=1, power=True, cpu_sample=1, ref_per_step=1,
                         desc="1 object, N_t=1000, N_f=1e5 on [0.1,10) c/d, full power + argmax"),
    "single_large": dict(kind="single", top_k=1, power=True, cpu_sample=1, ref_per_step=1,
                         desc="1 object, N_t=1e5, N_f=1e6 on [0.05,25) c/d, full power + argmax"),
}


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


DEFAULT_WORKLOAD = "ragged_lognormal"
CHECKPOINT = os.path.join(ROOT, "paper_2105_04006_gb300", "weights", "proposer_survey.npz")
LEARNED_N_OBJ = 100_000      # inference set of the learned path (survey-shaped, N_f = 1e5)


def make_workload(name, rank, n_obj=None):
    seed = synth.SEEDS[name] + 1_000_003 * rank
    kw = {"n_obj": n_obj} if n_obj else {}
    return synth.by_name(name, seed=seed, **kw)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.rows = []
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu_index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.first = threading.Event()
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        # nvidia-smi's start-up (NVML initialisation) can hold up the GPU work
        # launched meanwhile for about a second: the timed region starts only
        # after its first sample has arrived
        self.first.wait(timeout=10.0)
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [x.strip() for x in line.split(",")]))
            self.first.set()
        self.first.set()

    def mark(self, which):
        if which == 0:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [r for (ts, r) in self.rows if self.t0 - 0.25 <= ts <= self.t1 + 0.25 and len(r) >= 9]
        if not rows:
            rows = [r for (_, r) in self.rows if len(r) >= 9]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(power) if power else None}


def source_hash():
    h = hashlib.sha256()
    for f in ("lsp_main_impl.cuh", "lsp_common.cuh", "lsp_main_f32.cu"):
        with open(os.path.join(ROOT, "paper_2105_04006_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(workload, src_hash):
    """DRAM bytes per main-kernel launch from the committed ncu summary, if it is current."""
    path = os.path.join(ROOT, "profiles", "main_kernel_traffic.md")
    if not os.path.exists(path):
        return None
    for line in open(path):
        if line.startswith("| " + workload + " |"):
            cells = [c.strip() for c in line.strip().strip("|").split("|")]
            # | workload | source hash | bytes per launch (full workload) | ...
            if len(cells) >= 3 and cells[1] == src_hash:
                try:
                    return float(cells[2])
                except ValueError:
                    return None
    return None


# ------------------------------------------------------------- CPU baseline
def parity_vs_oracle(ref, peaks_np, top_k, power_np=None, precision="fp32"):
    """This run's results against the oracle's on the CPU-baseline sample."""
    tol = 1e-4 if precision == "fp32" else 1e-10
    if ref is None:
        return None
    if ref["kind"] == "single":
        if power_np is None:
            return None
        err = float(np.max(np.abs(power_np.reshape(-1)[ref["k"]].astype(np.float64) - ref["power"])))
        return {"compared": f"P_n at {ref['k'].size} sampled frequencies", "max_abs_err": err,
                "tolerance": tol, "within": err <= tol}
    first = peaks_np.reshape(-1, top_k)[ref["objects"], 0]
    dk = np.abs(first["idx"].astype(np.int64) - ref["arg_idx"].astype(np.int64))
    err = float(np.max(np.abs(first["power"] - ref["arg_pow"])))
    return {"compared": f"first maximum of {dk.size} sampled objects", "argmax_within_1_bin": float(np.mean(dk <= 1)),
            "argmax_exact": float(np.mean(dk == 0)), "max_abs_err_peak_power": err, "tolerance": tol}


def cpu_baseline(b, n_sample, top_k):
    import oracle
    oracle.build()
    g = b.grid
    if b.n_obj == 1:
        # one object: an evenly spaced subset of its frequencies (about 4e9 pairs)
        n_sel = int(min(g.n_f, max(1000, 4e9 // max(1, b.t.size))))
        ks = np.linspace(0, g.n_f - 1, n_sel).astype(np.int64)
        t0 = time.perf_counter()
        p_orc, _ = oracle.lsp_single(b.t, b.y.astype(np.float32).astype(np.float64), g.f_min, g.f_max, g.n_f,
                                     k_sel=ks)
        dt = time.perf_counter() - t0
        cpu_baseline.ref = {"kind": "single", "k": ks, "power": p_orc}
        frac = n_sel / g.n_f
        pairs = b.t.size * n_sel
        what = ("the whole object" if n_sel == g.n_f else
                f"{n_sel} of the object's {g.n_f} frequencies, extrapolated to the whole object")
        t0 = time.perf_counter()
        oracle.fp32_single(b.t, b.y.astype(np.float32).astype(np.float64), g.f_min, g.f_max, g.n_f, ks)
        dt32 = time.perf_counter() - t0
        return {"value": frac / dt, "unit": "objects/s", "cores": oracle.num_threads(), "kind": "oracle",
                "sample": f"{what} ({pairs:.3g} pairs, FP64 two-scan Eq. 1-2), {dt:.1f} s",
                "pairs_per_s": pairs / dt,
                "fp32_cpu": {"value": frac / dt32, "pairs_per_s": pairs / dt32, "seconds": dt32,
                             "what": "the same sample, two-scan Eq. 1-2 in FP32 (the paper's lsp-c FP32 mode)"}}
    n_sample = min(n_sample, b.n_obj)
    idx = np.linspace(0, b.n_obj - 1, n_sample).astype(np.int64)
    sub, what = b.subset(idx), f"{n_sample} objects evenly spaced over the batch"
    t0 = time.perf_counter()
    res = oracle.lsp_batch(sub.t, sub.y.astype(np.float32).astype(np.float64), sub.offsets, g.f_min, g.f_max,
                           g.n_f, top_k=top_k, return_power=False)
    dt = time.perf_counter() - t0
    cpu_baseline.ref = {"kind": "batch", "objects": idx, "arg_idx": res["arg_idx"], "arg_pow": res["arg_pow"]}
    t0 = time.perf_counter()
    oracle.fp32_batch_argmax(sub.t, sub.y.astype(np.float32).astype(np.float64), sub.offsets, g.f_min, g.f_max,
                             g.n_f)
    dt32 = time.perf_counter() - t0
    return {"value": sub.n_obj / dt, "unit": "objects/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{what} ({sub.pairs:.3g} pairs, FP64 two-scan Eq. 1-2), {dt:.1f} s",
            "pairs_per_s": sub.pairs / dt,
            "fp32_cpu": {"value": sub.n_obj / dt32, "pairs_per_s": sub.pairs / dt32, "seconds": dt32,
                         "what": "the same sample, two-scan Eq. 1-2 in FP32 (the paper's lsp-c FP32 mode)"}}


def run_reference(args, w, name):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    b = make_workload(name, 0, args.n_obj)
    per = w["ref_per_step"]
    g = b.grid
    steps_t = []

    def step(i):
        if b.n_obj == 1:
            n_sel = int(min(g.n_f, max(1000, 2e9 // max(1, b.t.size))))
            ks = np.linspace(0, g.n_f - 1, n_sel).astype(np.int64)
            t0 = time.perf_counter()
            oracle.lsp_single(b.t, b.y.astype(np.float32).astype(np.float64), g.f_min, g.f_max, g.n_f,
                              k_sel=ks)
            return time.perf_counter() - t0, n_sel / g.n_f
        else:
            lo = (i * per) % max(1, b.n_obj - per)
            sub = b.subset(np.arange(lo, lo + per))
        t0 = time.perf_counter()
        oracle.lsp_batch(sub.t, sub.y.astype(np.float32).astype(np.float64), sub.offsets, g.f_min, g.f_max,
                         g.n_f, top_k=w["top_k"], return_power=w["power"])
        return time.perf_counter() - t0, sub.n_obj

    for i in range(args.warmup):
        step(i)
    n_done = 0
    for i in range(args.steps):
        dt, n = step(args.warmup + i)
        steps_t.append(dt)
        n_done += n
    total = sum(steps_t)
    value = n_done / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "objects/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": name, "shape": w["desc"],
                                        "sample_per_step": (f"{per} objects" if b.n_obj > 1 else
                                                            "a frequency subsample of the object, extrapolated")},
        "cpu_baseline": {"value": value, "unit": "objects/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"{per if b.n_obj > 1 else 1} objects per step, {args.steps} steps"},
        "e2e": {"value": value, "unit": "objects/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------- GPU arm
GLS_OPS_PER_PAIR = 11  # generalized periodogram, rotation form: 4 (rotation) + 7 (u c, u s, w c, w s, w c, w c c, w c s)


def run_gls(args, w, name):
    """The generalized periodogram (Section 4.11) on a batch workload with seeded
    photometric errors dy ~ U[0.02, 0.3]: objects/s through lsp_batch_gls,
    its roofline against the 11-operation rotation form, the end-to-end time
    from pinned host buffers, the oracle's weighted least squares on a sample
    and the run's error against it."""
    import ctypes
    import torch
    import paper_2105_04006_gb300 as lsp
    import oracle

    rank, world, local = dist_env()
    if world > 1:
        raise SystemExit("--gls runs on one GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    b = make_workload(name, rank, args.n_obj)
    single = b.n_obj == 1  # lsp_periodogram_gls, split over the observations
    g = lsp.Grid(b.grid.f_min, b.grid.f_max, b.grid.n_f)
    fp64 = args.precision == "fp64"
    ydt = np.float64 if fp64 else np.float32
    dy = np.random.default_rng(synth.SEEDS[name] + 7).uniform(0.02, 0.3, b.t.size).astype(ydt)
    yv = b.y.astype(ydt)
    t = torch.tensor(b.t, dtype=torch.float64, device=dev)
    y = torch.tensor(yv, device=dev)
    e = torch.tensor(dy, device=dev)
    off = torch.tensor(b.offsets, dtype=torch.int64, device=dev)
    kw = {}
    if args.config:  # k_reseed,freqs_per_thread,block_threads[,obs_split] for the generalized kernels
        kw = dict(zip(("k_reseed", "freqs_per_thread", "block_threads", "obs_split"),
                      (int(v) for v in args.config.split(",")[:4])))
    opts = lsp.make_opts(precision=args.precision, top_k=w["top_k"], **kw)
    ws = torch.empty(max(lsp.workspace_size_gls(b.n_obj, b.t.size, g, opts), 256), dtype=torch.uint8, device=dev)
    peaks = torch.empty(b.n_obj * w["top_k"] * 40, dtype=torch.uint8, device=dev)
    # the full periodogram into HBM where the workload asks for it
    power = (torch.empty((b.n_obj, g.n_f), dtype=torch.float64 if fp64 else torch.float32, device=dev)
             if w["power"] else None)
    pw = ctypes.c_void_p(power.data_ptr()) if power is not None else None
    L = lsp.lib()
    P = ctypes.c_void_p

    def call(tp, yp, ep, op, pk):
        if single:
            st = L.lsp_periodogram_gls(P(tp), P(yp), P(ep), b.t.size, ctypes.byref(g), ctypes.byref(opts), pw,
                                       P(pk), P(ws.data_ptr()), ws.numel(), lsp._stream_handle(dev))
        else:
            st = L.lsp_batch_gls(P(tp), P(yp), P(ep), P(op), b.n_obj, b.t.size, ctypes.byref(g),
                                 ctypes.byref(opts), pw, P(pk), P(ws.data_ptr()), ws.numel(),
                                 lsp._stream_handle(dev))
        if st:
            raise lsp.LSPError(st, L.lsp_last_error().decode())

    run = lambda: call(t.data_ptr(), y.data_ptr(), e.data_ptr(), off.data_ptr(), peaks.data_ptr())
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0]
    clk = ClockSampler(gpu_index)
    clk.start()
    clk.mark(0)
    ms = []
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        run()
        c.record()
        c.synchronize()
        ms.append(a.elapsed_time(c))
    clk.mark(1)
    clocks = clk.stop()
    # end to end: inputs copied from pinned host memory, peaks copied back, every step
    th, yh, eh = (torch.from_numpy(x).pin_memory() for x in (b.t, yv, dy))
    oh = torch.from_numpy(b.offsets).pin_memory()
    pk_h = torch.empty(peaks.numel(), dtype=torch.uint8).pin_memory()
    td, yd, ed, od = (torch.empty_like(x, device=dev) for x in (th, yh, eh, oh))
    e2e_ms = []
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for dst, src in ((td, th), (yd, yh), (ed, eh)) + (() if single else ((od, oh),)):
            dst.copy_(src, non_blocking=True)
        call(td.data_ptr(), yd.data_ptr(), ed.data_ptr(), od.data_ptr(), peaks.data_ptr())
        pk_h.copy_(peaks, non_blocking=True)
        c.record()
        c.synchronize()
        e2e_ms.append(a.elapsed_time(c))
    step = statistics.mean(ms)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_mhz = (clocks or {}).get("sm_mhz") or 0.0
    achieved = b.pairs / (step / 1e3) / 1e9
    if fp64:  # FP64: against the measured DFMA rate
        peak = lsp.probe_fma_rates(dev)["f64"] / GLS_OPS_PER_PAIR / 1e9
        basis = f"measured DFMA rate / {GLS_OPS_PER_PAIR} ops per pair; achieved over whole steps"
    else:
        peak = n_sm * 128 * clk_mhz * 1e6 / GLS_OPS_PER_PAIR / 1e9 if clk_mhz else None
        basis = (f"{n_sm} SMs x 128 FP32 lanes x sampled SM clock / {GLS_OPS_PER_PAIR} ops per pair (the "
                 "generalized sums in the rotation form); achieved over whole steps")
    cpu = parity = None
    if not args.no_cpu and single:
        # a window of frequencies around the GPU's peak, timed and extrapolated
        oracle.build()
        first = lsp.peaks_to_numpy(peaks)[0]
        half = 1000
        k_lo = max(0, min(int(first["idx"]) - half, g.n_f - 2 * half))
        m = min(2 * half, g.n_f)
        t0 = time.perf_counter()
        res = oracle.gls_batch(b.t, yv.astype(np.float64), dy.astype(np.float64), b.offsets, g.f_min + k_lo * b.grid.df,
                               g.f_min + (k_lo + m) * b.grid.df, m, return_power=power is not None)
        dt = time.perf_counter() - t0
        cpu = {"value": (m / g.n_f) / dt, "unit": "objects/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"{m} of the {g.n_f} frequencies ({b.t.size * m:.3g} pairs, FP64 weighted 3-parameter "
                         f"least squares per frequency) in {dt:.1f} s, extrapolated to the whole grid"}
        dk = abs(int(first["idx"]) - (k_lo + int(res["arg_idx"][0])))
        parity = {"compared": f"first maximum against the oracle's maximum over {m} frequencies around it",
                  "argmax_within_1_bin": float(dk <= 1), "argmax_exact": float(dk == 0),
                  "max_abs_err_peak_power": float(abs(first["power"] - res["arg_pow"][0])),
                  "tolerance": 1e-10 if fp64 else 1e-4}
        if power is not None:
            win = power[0, k_lo:k_lo + m].double().cpu().numpy()
            parity["max_abs_err_window_power"] = float(np.max(np.abs(win - res["power"][0])))
    elif not args.no_cpu:
        oracle.build()
        n_sample = min(w["cpu_sample"] // 2, b.n_obj)
        idx = np.linspace(0, b.n_obj - 1, n_sample).astype(np.int64)
        sub = b.subset(idx)
        sub_dy = np.concatenate([dy[b.offsets[o]:b.offsets[o + 1]] for o in idx]).astype(np.float64)
        t0 = time.perf_counter()
        res = oracle.gls_batch(sub.t, sub.y.astype(ydt).astype(np.float64), sub_dy, sub.offsets, g.f_min, g.f_max,
                               g.n_f, return_power=False)
        dt = time.perf_counter() - t0
        cpu = {"value": sub.n_obj / dt, "unit": "objects/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"{n_sample} objects evenly spaced over the batch ({sub.pairs:.3g} pairs, FP64 weighted "
                         f"3-parameter least squares per frequency), {dt:.1f} s"}
        first = lsp.peaks_to_numpy(peaks).reshape(-1, w["top_k"])[idx, 0]
        dk = np.abs(first["idx"].astype(np.int64) - res["arg_idx"])
        parity = {"compared": f"first maximum of {n_sample} sampled objects",
                  "argmax_within_1_bin": float(np.mean(dk <= 1)), "argmax_exact": float(np.mean(dk == 0)),
                  "max_abs_err_peak_power": float(np.max(np.abs(first["power"] - res["arg_pow"]))),
                  "tolerance": 1e-10 if fp64 else 1e-4}
    h2d = b.t.size * 8 + yv.nbytes + dy.nbytes + (0 if single else b.offsets.nbytes)
    print(json.dumps({
        "impl": "gb300", "metric": METRIC + " (generalized periodogram)", "value": b.n_obj / (step / 1e3),
        "unit": "objects/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64" if fp64 else "f32",
        "data": "synthetic",
        "config": {"workload": name + "+gls", "shape": w["desc"] + ", dy ~ U[0.02, 0.3]", "n_obj": b.n_obj,
                   "total_nt": int(b.t.size), "n_f": g.n_f, "l2": "flushed between steps (256 MiB write)",
                   "kernel": "main_f32_packed_gls" if not fp64 else "main_f64_gls", "options": kw},
        "pairs_per_s": achieved * 1e9,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gpair/s",
                     "frac": achieved / peak if peak else None, "traffic": None,
                     "peak_basis": basis},
        "cpu_baseline": cpu, "parity_vs_oracle": parity,
        "e2e": {"value": b.n_obj / (statistics.mean(e2e_ms) / 1e3), "unit": "objects/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(peaks.numel()), "ms_per_step": statistics.mean(e2e_ms)},
        "gpu_launches": None, "clocks": clocks}), flush=True)
    return 0


def run_periodogram_return(args, w, name):
    """Section 3.5's transfer step on GB300: the full periodogram of a workload
    returned to the host by each route the library offers, device time per step
    (CUDA events on the launching stream, median of the steps)."""
    import torch
    import paper_2105_04006_gb300 as lsp

    rank, world, local = dist_env()
    if world > 1:
        raise SystemExit("--periodogram-return runs on one GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    b = make_workload(name, rank, args.n_obj)
    g = lsp.Grid(b.grid.f_min, b.grid.f_max, b.grid.n_f)
    t = torch.tensor(b.t, dtype=torch.float64, device=dev)
    y = torch.tensor(b.y.astype(np.float32), device=dev)
    off = torch.tensor(b.offsets, dtype=torch.int64, device=dev) if b.n_obj > 1 else None
    plan = lsp.Plan(b.n_obj, b.t.size, g)
    if not args.no_tune:
        plan.autotune(t, y, off, cache_path=os.path.join(ROOT, "paper_2105_04006_gb300", "_build", "tune_cache.jsonl"))
    shape = (b.n_obj, g.n_f)
    p_dev = torch.empty(shape, dtype=torch.float32, device=dev)
    p_pin = torch.empty(shape, dtype=torch.float32).pin_memory()
    p_pag = torch.from_numpy(np.empty(shape, dtype=np.float32))
    peaks = plan.peaks_buffer(dev)
    t_h = torch.from_numpy(np.ascontiguousarray(b.t)).pin_memory()
    y_h = torch.from_numpy(b.y.astype(np.float32)).pin_memory()
    off_h = torch.from_numpy(np.ascontiguousarray(b.offsets)).pin_memory() if off is not None else None
    pk_h = np.empty(b.n_obj, dtype=lsp.PEAK_DTYPE)

    def host(parts, out):
        def fn():
            plan.set_host_parts(parts)
            plan.execute_host(t_h, y_h, off_h, power=out, peaks=pk_h)
        return fn

    routes = {
        "peaks only (no periodogram)": lambda: plan.execute(t, y, off, peaks=peaks),
        "periodogram into HBM": lambda: plan.execute(t, y, off, power=p_dev, peaks=peaks),
        "into HBM, then copy to pinned host memory":
            lambda: (plan.execute(t, y, off, power=p_dev, peaks=peaks), p_pin.copy_(p_dev, non_blocking=True)),
        "into HBM, then copy to pageable host memory":
            lambda: (plan.execute(t, y, off, power=p_dev, peaks=peaks), p_pag.copy_(p_dev)),
        "written by the kernels straight into pinned host memory":
            lambda: plan.execute(t, y, off, power=p_pin, peaks=peaks),
        "host entry point (inputs in, peaks out), one pass into pinned memory": host(1, p_pin),
    }
    for n in (2, 4, 8, 16):
        routes[f"host entry point, {n} object groups, copies overlapped, pinned"] = host(n, p_pin)
    routes["host entry point, 8 object groups, copies overlapped, pageable"] = host(8, p_pag)
    out = {}
    for label, fn in routes.items():
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            c.record()
            c.synchronize()
            ms.append(a.elapsed_time(c))
        out[label] = statistics.median(ms)
    nbytes = b.n_obj * g.n_f * 4
    same = bool(torch.equal(p_pin, p_dev.cpu())) and bool(torch.equal(p_pag, p_dev.cpu()))
    plan.set_host_parts(0)
    default_parts = plan.host_parts()
    plan.close()
    copy_ms = out["into HBM, then copy to pinned host memory"] - out["periodogram into HBM"]
    print(json.dumps({"impl": "gb300", "mode": "periodogram_return", "workload": name, "n_obj": b.n_obj,
                      "n_f": g.n_f, "periodogram_bytes": nbytes, "ms_per_step": out,
                      "copy_GB_per_s": nbytes / (copy_ms * 1e-3) / 1e9 if copy_ms > 0 else None,
                      "host_routes_equal_device": same, "default_host_parts": default_parts,
                      "timing": "device time per step, CUDA events, median; L2 not flushed"}), flush=True)
    return 0


def run_ablations(args, lsp, torch, plan, b, t, y, off, name, rank):
    """The paper's kernel comparisons on GB300 through the autotuner: every candidate
    configuration, including the ablation kernels (per-pair SFU or accurate sin/cos
    instead of the recurrence; observations read from global memory instead of shared
    memory tiles), timed on this workload and checked against the FP64 path."""
    import tempfile
    clocks_s = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", str(t.device.index or 0)).split(",")[0])
    clocks_s.start()
    clocks_s.mark(0)
    with tempfile.TemporaryDirectory() as td:
        cfg, trials = plan.autotune(t, y, off, cache_path=os.path.join(td, "tune.jsonl"), ablations=True,
                                    return_trials=True)
    clocks_s.mark(1)
    clocks = clocks_s.stop()
    pairs = b.pairs
    rows = []
    for tr in trials:
        c = tr["config"]
        kind = ("recurrence", "SFU sincos per pair", "accurate sincospif per pair")[c["trig"]]
        rows.append({"config": c, "trig": kind, "staging": ("shared", "global")[c["staging"]],
                     "ms_per_step": tr["ms"], "pairs_per_s": pairs / (tr["ms"] * 1e-3) if tr["ms"] > 0 else None,
                     "max_err_vs_fp64": tr["max_err"], "passed_gate": tr["passed"]})
    plan.close()
    if rank == 0:
        print(json.dumps({"impl": "gb300", "mode": "ablations", "workload": name, "n_obj": b.n_obj,
                          "total_nt": int(b.t.size), "n_f": b.grid.n_f, "chosen": cfg, "trials": rows,
                          "clocks": clocks}), flush=True)
    return 0


def learned_leg(args, dev, gpu_index, log=None):
    """The learned proposal path against the plain full grid on the same
    100000 survey-shaped objects (N_t 50..500, N_f = 1e5 on [0.24, 12) c/d):
    device time per step (CUDA events, L2 flushed), recovery of the full
    grid's period (first maximum within one bin) and the cost breakdown."""
    import torch
    import paper_2105_04006_gb300 as lsp
    from paper_2105_04006_gb300 import learned as L

    ckpt = args.checkpoint or CHECKPOINT
    if os.path.exists(ckpt):
        prop, meta = L.Proposer.load_npz(ckpt, dev)
        trained_on = f"{os.path.relpath(ckpt, ROOT)}: {meta.get('trained_on', 'committed network')}"
    else:  # no committed network: train one on a bounded set in this run
        n_train = args.n_train_inrun
        per, sets = 25_000, []
        for part in range((n_train + per - 1) // per):
            sets.append(L.labelled_set(min(per, n_train - part * per), dev, "learned_train", part))
        prop = L.Proposer(sets[0]["grid"].n_f, dev, seed=1)
        L.train(prop, sets, epochs=10, batch_size=1024, lr=2e-3)
        del sets
        trained_on = f"{n_train} learned_train curves labelled by lsp_batch, trained in this run (10 epochs)"
    b = synth.learned_set(LEARNED_N_OBJ, "learned_infer", 1000)
    g = lsp.Grid(b.grid.f_min, b.grid.f_max, b.grid.n_f)
    t = torch.tensor(b.t, dtype=torch.float64, device=dev)
    y = torch.tensor(b.y.astype(np.float32), device=dev)
    off = torch.tensor(b.offsets, dtype=torch.int64, device=dev)
    plan = lsp.Plan(b.n_obj, b.t.size, g)
    if not args.no_tune:  # the plain full grid at its fastest configuration
        plan.autotune(t, y, off, cache_path=os.path.join(ROOT, "paper_2105_04006_gb300", "_build",
                                                         "tune_cache.jsonl"))
    peaks_plain = plan.peaks_buffer(dev)
    path = L.LearnedPath(prop)
    out = {}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ms = []
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            c.record()
            c.synchronize()
            ms.append(a.elapsed_time(c))
        return statistics.mean(ms)

    def learned():
        out["peaks"], out["info"] = path(t, y, off, g)

    clk = ClockSampler(gpu_index)
    clk.start()
    clk.mark(0)
    ms_plain = timed(lambda: plan.execute(t, y, off, peaks=peaks_plain))
    ms_learned = timed(learned)
    clk.mark(1)
    clocks = clk.stop()
    # the same path as its parts, each timed alone: features, MLP + top-k
    # (the tcgen05 GEMMs), windowed refine + full-grid fallback
    x16 = L.featurize(t, y, off, g)
    cls = prop.propose(x16)
    stages = {"featurize_ms": timed(lambda: L.featurize(t, y, off, g)),
              "mlp_topk_ms": timed(lambda: prop.propose(x16)),
              "refine_fallback_ms": timed(lambda: L.refine(t, y, off, g, cls, prop.k_windows, prop.stop_power,
                                                           prop.fallback_power, prop.inconclusive_fallback))}
    del x16, cls
    full = lsp.peaks_to_numpy(peaks_plain)
    got = lsp.peaks_to_numpy(out["peaks"])
    info = out["info"].cpu().numpy()
    rounds = info & 255
    fb = (info & L.REFINE_FALLBACK) != 0
    ok = np.abs(got["idx"] - full["idx"]) <= 1
    pairs = float(np.sum(b.n_t * (rounds * L.WINDOW + fb * g.n_f)))
    cfg_plain = plan.config
    plan.close()
    return {"workload": "learned_infer", "shape": f"{b.n_obj} objects, N_t~U{{50..500}}, seasonal cadence, "
                                                  "N_f=1e5 on [0.24,12) c/d, windows of 2048 bins, "
                                                  f"top-{prop.k_windows} proposals, full-grid fallback below "
                                                  f"P_n {prop.fallback_power}",
            "value": b.n_obj / (ms_learned / 1e3), "unit": "objects/s", "ms_per_step": ms_learned,
            "plain": {"value": b.n_obj / (ms_plain / 1e3), "ms_per_step": ms_plain, "kernel_config": cfg_plain},
            "speedup_vs_plain": ms_plain / ms_learned,
            "recovery": float(ok.mean()), "recovered_of": int(ok.size),
            "fallback_fraction": float(fb.mean()), "mean_windows": float(rounds.mean()),
            "pair_fraction": pairs / float(b.pairs), "stop_power": prop.stop_power,
            "trained_on": trained_on, "entry_point": "lsp_propose_refine (one call per step)",
            "stages": stages,
            "steps": args.steps, "warmup": args.warmup, "l2": "flushed between steps (256 MiB write)",
            "clocks": clocks}


def run_mlp(args):
    """The proposal network's products on the tcgen05 tensor cores: forward
    passes of the survey network (512 -> 256 -> 256 -> 256 -> 98) on 20 000
    and 100 000 rows and loss + gradient at batches of 1024 and 4096, device
    time per call (CUDA events, L2 flushed), against the measured bf16 tensor
    peak and the HBM bytes the pass moves."""
    import torch
    from paper_2105_04006_gb300 import learned as L

    rank, world, local = dist_env()
    if world > 1:
        raise SystemExit("--mlp runs on one GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prop = L.Proposer(100_000, dev, seed=1)
    d = prop.dims
    macs = sum(a * b for a, b in [(d.in_dim, d.hidden)] + [(d.hidden, d.hidden)] * (d.n_hidden - 1)
               + [(d.hidden, d.n_classes)])
    macs_dx = macs - d.in_dim * d.hidden  # no input gradient for the first layer
    peaks = {}
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    tflops_peak, hbm_peak = peaks.get("bf16_tflops"), peaks.get("hbm_gbs")
    gen = torch.Generator(device="cpu").manual_seed(7)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ms = []
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            c.record()
            c.synchronize()
            ms.append(a.elapsed_time(c))
        return statistics.mean(ms)

    legs = []
    for rows in (20_000, 100_000):
        x16 = torch.randn(rows, d.in_dim, generator=gen).to(torch.bfloat16).to(dev)
        ms = timed(lambda: prop.forward(x16))
        flops = 2.0 * rows * macs
        hbm = rows * (2 * d.in_dim + 2 * 2 * d.hidden * d.n_hidden + 4 * d.n_classes)
        legs.append({"pass": "forward", "rows": rows, "ms": ms, "tflops": flops / ms / 1e9,
                     "frac_bf16_peak": flops / ms / 1e9 / tflops_peak if tflops_peak else None,
                     "hbm_bytes": hbm, "gbs": hbm / ms / 1e6,
                     "frac_hbm_peak": hbm / ms / 1e6 / hbm_peak if hbm_peak else None})
    for batch in (1024, 4096):
        x16 = torch.randn(batch, d.in_dim, generator=gen).to(torch.bfloat16).to(dev)
        lab = torch.randint(0, d.n_classes, (batch,), generator=gen, dtype=torch.int32).to(dev)
        ms = timed(lambda: prop.loss_grad(x16, lab))
        flops = 2.0 * batch * (2 * macs + macs_dx)
        legs.append({"pass": "loss_grad", "rows": batch, "ms": ms, "tflops": flops / ms / 1e9,
                     "frac_bf16_peak": flops / ms / 1e9 / tflops_peak if tflops_peak else None})
    line = {"impl": "gb300", "metric": "proposal-network GEMMs (tcgen05 + TMA): device ms per call",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "dtype": "bf16 x bf16 -> f32",
            "data": "synthetic", "config": {"workload": "mlp", "network": f"{d.in_dim}-{d.hidden}x{d.n_hidden}-"
                                                                        f"{d.n_classes}",
                                            "l2": "flushed between steps (256 MiB write)",
                                            "hbm_bytes": "forward: inputs read, hidden activations written "
                                                         "and read back, FP32 logits written"},
            "legs": legs, "peaks": {"bf16_tflops": tflops_peak, "hbm_gbs": hbm_peak}}
    print(json.dumps(line), flush=True)
    return 0


OTHER_LEGS = (("ragged_survey", "fp32"), ("single_small", "fp32"), ("single_small", "fp64"),
              ("single_large", "fp32"), ("single_large", "fp64"))


def other_leg(args, dev, name, precision, steps):
    """One more workload of the same metric, measured like the main line but
    compactly: autotuned plan, device time per step (L2 flushed), the main
    kernel's time and fraction of its bound, and the run's error against the
    oracle on a small sample (16 objects, or 200 frequencies of one object)."""
    import torch
    import paper_2105_04006_gb300 as lsp
    import oracle

    w = WORKLOADS[name]
    b = make_workload(name, 0)
    g = lsp.Grid(b.grid.f_min, b.grid.f_max, b.grid.n_f)
    fp64 = precision == "fp64"
    ydt = np.float64 if fp64 else np.float32
    t = torch.tensor(b.t, dtype=torch.float64, device=dev)
    y = torch.tensor(b.y.astype(ydt), device=dev)
    off = torch.tensor(b.offsets, dtype=torch.int64, device=dev) if b.n_obj > 1 else None
    power = (torch.empty((b.n_obj, g.n_f), dtype=torch.float64 if fp64 else torch.float32, device=dev)
             if w["power"] else None)
    plan = lsp.Plan(b.n_obj, b.t.size, g, top_k=w["top_k"], precision=precision)
    # the FP64 path on the 1e11-pair object takes 1.3 s a step: its default
    # configuration, no tuning
    tuned = not args.no_tune and not (fp64 and b.pairs > 1e10)
    if tuned:
        plan.autotune(t, y, off, cache_path=os.path.join(ROOT, "paper_2105_04006_gb300", "_build", "tune_cache.jsonl"))
    if fp64 and b.pairs > 1e10:
        steps = min(steps, 5)
    peaks = plan.peaks_buffer(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed(probe):
        # the step without the probe; the main kernel's time in a second pass
        # with it (its event nodes add to a short step and keep the kernels
        # from overlapping their launches)
        plan.enable_timing(probe)
        for _ in range(args.warmup):
            plan.execute(t, y, off, power=power, peaks=peaks)
        torch.cuda.synchronize()
        step_ms, main_ms = [], []
        for i in range(steps):
            flush.fill_(i & 0xFF)
            a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            plan.execute(t, y, off, power=power, peaks=peaks)
            c.record()
            c.synchronize()
            step_ms.append(a.elapsed_time(c))
            if probe:
                main_ms.append(plan.main_kernel_ms())
        return statistics.mean(step_ms), (statistics.mean(main_ms) if main_ms else None)

    st, _ = timed(False)
    _, mk = timed(True)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    achieved = b.pairs / (mk / 1e3) / 1e9
    if fp64:
        peak = lsp.probe_fma_rates(dev)["f64"] / OPS_PER_PAIR / 1e9
        basis = f"measured DFMA rate / {OPS_PER_PAIR} ops per pair"
    else:
        peak = n_sm * FP32_LANES_PER_SM * 2070e6 / OPS_PER_PAIR / 1e9
        basis = f"{n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2070 MHz / {OPS_PER_PAIR} ops per pair"
    # the run's own error against the oracle on a small sample
    oracle.build()
    tol = 1e-10 if fp64 else 1e-4
    yv = b.y.astype(ydt).astype(np.float64)
    if b.n_obj == 1:
        pw = power.reshape(-1).double().cpu().numpy()
        ks = np.unique(np.concatenate([np.linspace(0, g.n_f - 1, 200).astype(np.int64),
                                       [int(np.argmax(pw))]]))
        ref, _ = oracle.lsp_single(b.t, yv, g.f_min, g.f_max, g.n_f, k_sel=ks)
        par = {"compared": f"P_n at {ks.size} frequencies incl. the maximum", "max_abs_err": float(np.max(np.abs(
            pw[ks] - ref))), "tolerance": tol}
    else:
        idx = np.linspace(0, b.n_obj - 1, 16).astype(np.int64)
        sub = b.subset(idx)
        res = oracle.lsp_batch(sub.t, sub.y.astype(ydt).astype(np.float64), sub.offsets, g.f_min, g.f_max, g.n_f,
                               top_k=1)
        first = lsp.peaks_to_numpy(peaks).reshape(-1, w["top_k"])[idx, 0]
        dk = np.abs(first["idx"].astype(np.int64) - res["arg_idx"])
        par = {"compared": f"first maximum of {idx.size} objects", "argmax_within_1_bin": float(np.mean(dk <= 1)),
               "max_abs_err_peak_power": float(np.max(np.abs(first["power"] - res["arg_pow"]))), "tolerance": tol}
    out = {"workload": name, "precision": precision, "shape": w["desc"], "value": b.n_obj / (st / 1e3),
           "unit": "objects/s", "ms_per_step": st, "main_kernel_ms": mk, "pairs_per_s": b.pairs / (st / 1e3),
           "timing": "step without the timing probe; main kernel from a second pass with it",
           "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gpair/s",
                        "frac": achieved / peak, "peak_basis": basis},
           "kernel_config": plan.config, "autotuned": tuned, "gpu_launches_per_step": plan.kernel_count,
           "steps": steps,
           "parity_vs_oracle": par}
    plan.close()
    return out


def run_gpu(args, w, name):
    import torch
    import paper_2105_04006_gb300 as lsp

    rank, world, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    sharded = world > 1 and not args.replicas
    if sharded:
        # one batch, cut into N_t-balanced contiguous object ranges: rank r runs
        # its own slice (no exchange on the data path)
        from paper_2105_04006_gb300 import shard
        full = make_workload(name, 0, args.n_obj)
        ranges = shard.shard_ranges(full.offsets, world)
        o0, o1 = ranges[rank]
        b = full.subset(np.arange(o0, o1))
    else:
        b = make_workload(name, rank, args.n_obj)
    g = lsp.Grid(b.grid.f_min, b.grid.f_max, b.grid.n_f)
    fp64 = args.precision == "fp64"
    ydt = np.float64 if fp64 else np.float32
    t = torch.tensor(b.t, dtype=torch.float64, device=dev)
    y = torch.tensor(b.y.astype(ydt), device=dev)
    off = torch.tensor(b.offsets, dtype=torch.int64, device=dev) if b.n_obj > 1 else None
    power = (torch.empty((b.n_obj, g.n_f), dtype=torch.float64 if fp64 else torch.float32, device=dev)
             if w["power"] else None)
    plan = lsp.Plan(b.n_obj, b.t.size, g, top_k=w["top_k"], precision=args.precision)
    if args.ablations:
        return run_ablations(args, lsp, torch, plan, b, t, y, off, name, rank)
    if args.config:
        keys = ("k_reseed", "freqs_per_thread", "block_threads", "obs_split", "packed", "trig", "staging")
        plan.set_config(**dict(zip(keys, (int(v) for v in args.config.split(",")))))
    elif not args.no_tune:
        cache = os.path.join(ROOT, "paper_2105_04006_gb300", "_build", "tune_cache.jsonl")
        plan.autotune(t, y, off, cache_path=cache)
    plan.enable_timing(True)
    peaks = plan.peaks_buffer(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        plan.execute(t, y, off, power=power, peaks=peaks)
    barrier()
    gpu_index = (os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[local]
                 if os.environ.get("CUDA_VISIBLE_DEVICES") else str(local))
    clk = ClockSampler(gpu_index)
    clk.start()
    barrier()
    clk.mark(0)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    main_ms = []
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        ev[i][0].record()
        plan.execute(t, y, off, power=power, peaks=peaks)
        ev[i][1].record()
        main_ms.append(plan.main_kernel_ms())
    barrier()
    clk.mark(1)
    clocks = clk.stop()
    step_ms = [a.elapsed_time(c) for a, c in ev]
    total_s = torch.tensor([sum(step_ms) / 1e3], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(total_s, op=dist.ReduceOp.MAX)
    total_s = float(total_s.item())
    n_units = torch.tensor([b.n_obj], dtype=torch.float64, device=dev)  # objects this rank processed per step
    if dist is not None:
        dist.all_reduce(n_units)
    value = float(n_units.item()) * args.steps / total_s
    pairs = b.pairs
    gathered = None
    if sharded:  # the only exchange: every rank's peak records to rank 0
        gathered = shard.gather_peaks(lsp.peaks_to_numpy(peaks), ranges, rank, per_object=w["top_k"])

    # end to end through the host-buffer entry point (pinned host memory)
    th = torch.from_numpy(b.t).pin_memory()
    yh = torch.from_numpy(b.y.astype(ydt)).pin_memory()
    oh = torch.from_numpy(b.offsets).pin_memory() if b.n_obj > 1 else None
    ph = (torch.empty((b.n_obj, g.n_f), dtype=torch.float64 if fp64 else torch.float32).pin_memory()
          if w["power"] else None)
    pk_host = np.empty(b.n_obj * w["top_k"], dtype=lsp.PEAK_DTYPE)
    plan.enable_timing(False)
    plan.set_host_parts(args.host_parts)
    plan.execute_host(th, yh, oh, power=ph, peaks=pk_host)  # warm: allocates staging, captures
    barrier()
    e2e_ms = []
    clk_e2e = ClockSampler(gpu_index)
    clk_e2e.start()
    clk_e2e.mark(0)
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        plan.execute_host(th, yh, oh, power=ph, peaks=pk_host)
        c.record()
        c.synchronize()
        e2e_ms.append(a.elapsed_time(c))
    clk_e2e.mark(1)
    clocks_e2e = clk_e2e.stop()
    e2e_s = torch.tensor([sum(e2e_ms) / 1e3], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(e2e_s, op=dist.ReduceOp.MAX)
    e2e_value = float(n_units.item()) * args.steps / float(e2e_s.item())
    ysz = 8 if fp64 else 4
    h2d = th.numel() * 8 + yh.numel() * ysz + (oh.numel() * 8 if oh is not None else 0)
    d2h = pk_host.nbytes + (ph.numel() * ysz if ph is not None else 0)

    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    main_avg = statistics.mean(main_ms)
    achieved = pairs / (main_avg / 1e3) / 1e9
    clk_mhz = (clocks or {}).get("sm_mhz") or 0.0
    lanes = FP64_LANES_PER_SM if fp64 else FP32_LANES_PER_SM
    rates = lsp.probe_fma_rates(dev)  # measured pipe ceilings, outside the timed region
    if fp64:  # FP64: against the measured DFMA rate
        peak = rates["f64"] / OPS_PER_PAIR / 1e9
        basis = f"measured DFMA rate {rates['f64'] / 1e9:.0f} G/s (register-only probe) / {OPS_PER_PAIR} ops per pair"
    else:     # FP32: nominal lanes at the sampled SM clock
        peak = n_sm * lanes * clk_mhz * 1e6 / OPS_PER_PAIR / 1e9 if clk_mhz else None
        basis = f"{n_sm} SMs x {lanes} FP32 lanes x sampled SM clock / {OPS_PER_PAIR} ops per pair"
    peak_max = n_sm * lanes * 2070e6 / OPS_PER_PAIR / 1e9
    ceiling = (rates["f64"] if fp64 else rates["f32x2"]) / OPS_PER_PAIR / 1e9
    src = source_hash()
    traffic = recorded_traffic(name, src)

    line = None
    if rank == 0:
        bb = full if sharded else b  # rank 0 checks the whole job's results
        cpu = None if args.no_cpu else cpu_baseline(bb, w["cpu_sample"], w["top_k"])
        parity = None
        if cpu is not None:  # this run's own results against the oracle on the same sample
            pk_np = gathered if sharded else lsp.peaks_to_numpy(peaks)
            pw_np = power.cpu().numpy() if (power is not None and not sharded) else None
            parity = parity_vs_oracle(getattr(cpu_baseline, "ref", None), pk_np, w["top_k"], pw_np, args.precision)
        learned = None
        if args.learned and world == 1 and not fp64:
            learned = learned_leg(args, dev, gpu_index)
        others = None
        if args.others and world == 1 and name == DEFAULT_WORKLOAD and not fp64:
            clk_o = ClockSampler(gpu_index)
            clk_o.start()
            clk_o.mark(0)
            others = [other_leg(args, dev, n, pr, min(args.steps, 10)) for n, pr in OTHER_LEGS]
            clk_o.mark(1)
            others = {"legs": others, "clocks": clk_o.stop(),
                      "note": "the other workloads of the same metric, each autotuned and timed on its own"}
        line = {
            "impl": "gb300", "metric": METRIC, "value": value, "unit": "objects/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms),
            "higher_is_better": True, "scaling": "strong" if sharded else "weak", "vs_baseline": None,
            "dtype": "f64" if fp64 else "f32", "data": "synthetic",
            "config": {"workload": name, "shape": w["desc"], "n_obj": int(n_units.item()),
                       "total_nt": int(bb.t.size), "n_f": g.n_f,
                       "parallelism": (f"objects sharded over {world} ranks by N_t" if sharded else
                                       f"{world} independent replicas" if world > 1 else "1 GPU"),
                       "precision": "fp64" if fp64 else "fp32 sums, fp64/fixed-point phase",
                       "l2": "flushed between steps (256 MiB write)", "kernel_config": plan.config},
            "pairs_per_s": world * pairs * args.steps / total_s,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gpair/s",
                         "frac": (achieved / peak) if peak else None, "traffic": traffic,
                         "kernel": "main trig-sum kernel", "main_kernel_ms": main_avg,
                         "peak_basis": basis, "peak_nominal_at_max_clock": peak_max,
                         "measured_fma_rates_per_s": rates,
                         "frac_of_measured_pipe_ceiling": achieved / ceiling,
                         "kernel_ops_per_pair": KERNEL_OPS_PER_PAIR,
                         "frac_note": (f"frac counts {OPS_PER_PAIR} FP32 operations per pair (the rotation "
                                       f"recurrence's algorithmic work); the kernel issues {KERNEL_OPS_PER_PAIR}, "
                                       "so its FP32 pipe is busy frac x 6/8 (pipe_busy_with_kernel_ops)"),
                         "pipe_busy_with_kernel_ops": (achieved * KERNEL_OPS_PER_PAIR / OPS_PER_PAIR / peak)
                         if (peak and not fp64) else achieved * KERNEL_OPS_PER_PAIR / OPS_PER_PAIR / ceiling,
                         "source_hash": src},
            "cpu_baseline": cpu,
            "parity_vs_oracle": parity,
            "e2e": {"value": e2e_value, "unit": "objects/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "ms_per_step": statistics.mean(e2e_ms),
                    "host_parts": plan.host_parts(power=ph is not None),
                    "ms_min": min(e2e_ms), "ms_max": max(e2e_ms), "clocks": clocks_e2e},
            "gpu_launches": plan.kernel_count * args.steps,
            "clocks": clocks,
            "learned": learned,
            "other_workloads": others,
        }
    plan.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ learned vs plain
def run_learned(args):
    """Train the proposal network (unless the checkpoint exists), write it, and
    time the learned path against the plain full grid (the learned leg)."""
    import torch
    from paper_2105_04006_gb300 import learned as L

    rank, world, local = dist_env()
    if world > 1:
        raise SystemExit("--workload learned runs on one GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ckpt = args.checkpoint or CHECKPOINT
    train_s = None
    if not os.path.exists(ckpt):
        t0 = time.perf_counter()
        per, sets = 25_000, []
        for part in range((args.n_train + per - 1) // per):
            sets.append(L.labelled_set(min(per, args.n_train - part * per), dev, "learned_train", part))
        prop = L.Proposer(sets[0]["grid"].n_f, dev, seed=1)
        hist = L.train(prop, sets, epochs=10, batch_size=1024, lr=2e-3)
        del sets
        train_s = time.perf_counter() - t0
        os.makedirs(os.path.dirname(os.path.abspath(ckpt)), exist_ok=True)
        prop.save_npz(ckpt, trained_on=(f"{args.n_train} learned_train curves (seeds disjoint from the inference "
                                        "set) labelled by lsp_batch, 10 epochs of AdamW, batch 1024, "
                                        f"lr 2e-3 cosine; final loss {hist[-1]:.4f}"))
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0]
    leg = learned_leg(args, dev, gpu_index)
    line = {"impl": "gb300", "metric": METRIC, "value": leg["value"], "unit": "objects/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": leg["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": "learned", "shape": leg["shape"]},
            "training_s": train_s, "checkpoint": os.path.relpath(ckpt, ROOT), "learned": leg}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["learned"], default=DEFAULT_WORKLOAD)
    ap.add_argument("--n-train", type=int, default=1_000_000, help="learned workload: training curves")
    ap.add_argument("--checkpoint", default=None,
                    help="proposer network (.npz) to load (learned leg, learned workload) or to write (learned "
                         "workload, when it does not exist); default: the committed network")
    ap.add_argument("--no-learned", dest="learned", action="store_false",
                    help="skip the learned-vs-plain leg of the default run")
    ap.add_argument("--n-train-inrun", type=int, default=200_000,
                    help="learned leg without a committed network: training curves generated in the run")
    ap.add_argument("--no-others", dest="others", action="store_false",
                    help="skip the compact legs of the other workloads in the default run")
    ap.add_argument("--replicas", action="store_true",
                    help="under torchrun: every rank runs its own batch (weak scaling) instead of a shard of one")
    ap.add_argument("--no-tune", action="store_true", help="use the default kernel configuration")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--config", default=None,
                    help="force a kernel configuration: k_reseed,freqs_per_thread,block_threads,obs_split,packed"
                         "[,trig,staging]")
    ap.add_argument("--periodogram-return", action="store_true",
                    help="time the routes that return a full periodogram to the host (Section 3.5)")
    ap.add_argument("--mlp", action="store_true",
                    help="time the proposal network's tensor-core GEMMs (forward and loss + gradient)")
    ap.add_argument("--gls", action="store_true",
                    help="the generalized periodogram (photometric errors, floating mean) on a batch workload")
    ap.add_argument("--ablations", action="store_true",
                    help="time every autotuner candidate, including the trig/staging ablation kernels, and print "
                         "them (one JSON line) instead of the benchmark")
    ap.add_argument("--host-parts", type=int, default=0,
                    help="object groups of the e2e leg's host entry point (0: the library's rule, 1: one pass)")
    ap.add_argument("--n-obj", type=int, default=None,
                    help="objects in a batch workload (default: the workload's own count)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.mlp:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the proposal network has no CPU reference arm"}))
            return 0
        return run_mlp(args)
    if args.workload == "learned":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the learned stage has no CPU reference arm"}))
            return 0
        return run_learned(args)
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w, args.workload)
    if args.gls:
        return run_gls(args, w, args.workload)
    if args.periodogram_return:
        return run_periodogram_return(args, w, args.workload)
    return run_gpu(args, w, args.workload)


if __name__ == "__main__":
    sys.exit(main())
