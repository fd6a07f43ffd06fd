#!/usr/bin/env python
"""Benchmark: TSMTTSM percent of roofline over the width sweep at K = 2^24.

One step = the whole sweep of plain-FP64 TSMTTSM calls (real with op T and
complex with op C, alpha = 1, beta = 0) at K = 2^24 rows for
M = N in {1, 2, 4, 8, 16, 32, 64} and (M, N) in {(1,64), (64,1), (8,32),
(32,8)}: 22 kernel launches on inputs already resident in HBM.

Roofline per call (Sec. 1.3, Eq. 1): flops = 2MNK (real) or 8MNK (complex),
bytes = 8c(MK + NK + MN) (c = 2 for complex), P_max = min(I * b_s, P_fp64)
with b_s the measured HBM bandwidth (MEASURED_PEAKS.json) and P_fp64 the
larger of the nominal GB300 FP64 rate and the rate the DFMA probe measures
live.  The reported value is whole-sweep efficiency:
100 * sum(ideal time) / sum(measured time).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       python bench.py --case c64:64x64 --k 1048576   (one kernel, for profiling)
"""

import argparse
import ctypes
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

K_FULL = 1 << 24
SQUARE = (1, 2, 4, 8, 16, 32, 64)
OFFDIAG = ((1, 64), (64, 1), (8, 32), (32, 8))
SWEEP = [(c, m, n) for c in (False, True) for (m, n) in [(w, w) for w in SQUARE] + list(OFFDIAG)]
FP64_NOMINAL_GFLOPS = 1250.0   # GB300 FP64 (vector and tensor), per GPU
HBM_FALLBACK_GBS = 6800.0
WORKLOAD = ("TSMTTSM FP64 sweep, K=2^24, real (op T) + complex (op C), M=N in {1,2,4,8,16,32,64} "
            "+ (M,N) in {(1,64),(64,1),(8,32),(32,8)}, alpha=1, beta=0, row-major, ld=width, "
            "uniform(-1,1) SplitMix64 inputs (A seed 0, B seed 1)")


def model(cplx, M, N, K):
    """(flops, bytes) of one TSMTTSM call with beta = 0 (Eq. 1 of the paper,
    complex: 4x flops, 2x bytes)."""
    c = 2 if cplx else 1
    flops = 2.0 * M * N * K * (4 if cplx else 1)
    nbytes = 8.0 * c * (M * K + N * K + M * N)
    return flops, nbytes


def ideal_seconds(cplx, M, N, K, bw_gbs, p64_gflops):
    flops, nbytes = model(cplx, M, N, K)
    return max(nbytes / (bw_gbs * 1e9), flops / (p64_gflops * 1e9))


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        loaded = [s for s in sm if s and s > 0.5 * (max(sm) if sm else 1)]
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            for i, n in enumerate(names):
                if r[5 + i].lower().startswith("active"):
                    reasons.add(n)
        power = [num(r[3]) for r in rows if num(r[3]) is not None]
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows), "power_w_max": max(power) if power else None}


# ------------------------------------------------------------------ helpers

def _kernel_source_hash(variant_name):
    """Hash of the sources that define a variant's kernel: the hand-written
    FP64 family or the generator, plus their shared epilogue and header."""
    h = hashlib.sha256()
    pkg = os.path.join(ROOT, "paper_1905_03136_gb300")
    files = ["csrc/fp64_common.cuh", "csrc/tsm_internal.h"]
    files.append("codegen.py" if variant_name.startswith("gen_") else "csrc/kernels_fp64.cu")
    for name in files:
        with open(os.path.join(pkg, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic_for(variant_name, cfg_key):
    """DRAM bytes per launch from a committed ncu capture, if it was taken on
    the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    e = d.get(cfg_key)
    if not e or e.get("source_hash") != _kernel_source_hash(variant_name) or e.get("variant") != variant_name:
        return None
    return e.get("dram_bytes_per_launch")


def _views(flatA, flatB, cplx, M, N, K):
    import torch
    c = 2 if cplx else 1
    a = flatA[: K * M * c]
    b = flatB[: K * N * c]
    if cplx:
        a = a.view(torch.complex128)
        b = b.view(torch.complex128)
    return a.view(K, M), b.view(K, N)


def cpu_oracle_sweep(K_sample, K_full, bw, p64):
    """Times the CPU oracle (single thread, as it stands) on the first
    K_sample rows of every sweep configuration; returns (value, seconds,
    per-config list) with times scaled linearly to K_full rows."""
    import numpy as np
    import oracle
    import synth
    total_ideal = 0.0
    total_cpu = 0.0
    wall = 0.0
    for (cplx, M, N) in SWEEP:
        A = synth.block_vector(synth.SEED_A, K_sample, M, complex_=cplx)
        B = synth.block_vector(synth.SEED_B, K_sample, N, complex_=cplx)
        C = np.zeros((M, N), dtype=A.dtype)
        t0 = time.perf_counter()
        oracle.tsmttsm("C" if cplx else "T", M, N, K_sample, 1.0, A, M, B, N, 0.0, C, N)
        dt = time.perf_counter() - t0
        wall += dt
        total_cpu += dt * K_full / K_sample
        total_ideal += ideal_seconds(cplx, M, N, K_full, bw, p64)
    return 100.0 * total_ideal / total_cpu, wall


# ------------------------------------------------------------------ arms

def run_reference(args, bw, bw_src):
    """The oracle as the reference arm: each step a bounded sample of the
    sweep on the host (single-threaded C oracle)."""
    p64 = FP64_NOMINAL_GFLOPS
    K_s = args.ref_rows
    for _ in range(args.warmup):
        cpu_oracle_sweep(K_s, K_FULL, bw, p64)
    vals, walls = [], []
    for _ in range(args.steps):
        v, w = cpu_oracle_sweep(K_s, K_FULL, bw, p64)
        vals.append(v)
        walls.append(w)
    value = statistics.mean(vals)
    sample = "first %d of 2^24 rows of each of the 22 sweep configurations, times scaled x%d" % (K_s, K_FULL // K_s)
    line = {"impl": "reference", "metric": "TSMTTSM % of roofline vs width, K=2^24", "value": value,
            "unit": "% of roofline", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(walls), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (SplitMix64 seeded)",
            "config": {"workload": WORKLOAD, "K": K_FULL, "parallelism": "replicas"},
            "cpu_baseline": {"value": value, "unit": "% of roofline", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "% of roofline", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "peaks": {"hbm_gbs": bw, "hbm_source": bw_src, "fp64_gflops": p64, "fp64_source": "nominal"}}
    print(json.dumps(line), flush=True)


def run_case(args):
    """One configuration, a few calls: the small case for ncu captures."""
    import torch
    import paper_1905_03136_gb300 as tsm
    tsm.load()
    kind, shape = args.case.split(":")
    M, N = (int(x) for x in shape.split("x"))
    cplx = kind == "c64"
    c = 2 if cplx else 1
    K = args.k
    fa = torch.empty(K * M * c, dtype=torch.float64, device="cuda")
    fb = torch.empty(K * N * c, dtype=torch.float64, device="cuda")
    tsm.fill_random(fa.view(1, -1), 0)
    tsm.fill_random(fb.view(1, -1), 1)
    A, B = _views(fa, fb, cplx, M, N, K)
    C = torch.zeros((M, N), dtype=A.dtype, device="cuda")
    for _ in range(args.steps):
        if args.split:
            from paper_1905_03136_gb300 import split
            split.tsmttsm_split(A, B, C, op="C" if cplx else "T")
        else:
            tsm.tsmttsm(A, B, C, op="C" if cplx else "T")
    torch.cuda.synchronize()
    print(json.dumps({"case": args.case, "K": K, "ok": True}))


def max_over_ranks(x, device=None):
    """The largest of every rank's x: the job's time is its slowest rank's
    (x itself when the process is not part of a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_ours(args, bw, bw_src):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_1905_03136_gb300 as tsm
    from paper_1905_03136_gb300 import probe
    tsm.load()
    dev = torch.device("cuda", local)
    K = K_FULL

    # Inputs: one flat buffer per operand, seeded once (outside timing).
    flatA = torch.empty(K * 128, dtype=torch.float64, device=dev)
    flatB = torch.empty(K * 128, dtype=torch.float64, device=dev)
    tsm.fill_random(flatA.view(K, 128), 0)
    tsm.fill_random(flatB.view(K, 128), 1)
    outs = {cfg: torch.zeros((cfg[1], cfg[2]), dtype=torch.complex128 if cfg[0] else torch.float64, device=dev)
            for cfg in SWEEP}
    views = {cfg: _views(flatA, flatB, cfg[0], cfg[1], cfg[2], K) for cfg in SWEEP}
    chosen = {cfg: tsm.choose(tsm.KIND_TSMTTSM, tsm.C64 if cfg[0] else tsm.R64, cfg[1], cfg[2], K) for cfg in SWEEP}
    names = {v["index"]: v["name"] for v in tsm.variants(tsm.KIND_TSMTTSM)}

    dfma = probe.fp64_peak(0)
    dmma = probe.fp64_peak(1)
    p64 = max(FP64_NOMINAL_GFLOPS, dfma, dmma)
    p64_src = "nominal" if p64 == FP64_NOMINAL_GFLOPS else ("measured DFMA probe" if p64 == dfma else
                                                             "measured DMMA probe")

    stream = torch.cuda.current_stream()

    def step(record=None):
        for cfg in SWEEP:
            A, B = views[cfg]
            if record is not None:
                record[cfg][0].record(stream)
            tsm.tsmttsm(A, B, outs[cfg], op="C" if cfg[0] else "T")
            if record is not None:
                record[cfg][1].record(stream)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()

    events = [{cfg: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for cfg in SWEEP} for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    t_start.record(stream)
    for s in range(args.steps):
        step(events[s])
    t_end.record(stream)
    torch.cuda.synchronize()
    clock_info = clocks.stop()
    if world > 1:
        dist.barrier()
    total_ms = t_start.elapsed_time(t_end)
    # Per-call times are medians over the steps: the first call of the first
    # timed step starts on an idle GPU and so also holds the host's launch
    # latency (the whole-step value above keeps it).
    per_cfg = {cfg: statistics.median(events[s][cfg][0].elapsed_time(events[s][cfg][1])
                                      for s in range(args.steps))
               for cfg in SWEEP}

    ideal = {cfg: ideal_seconds(cfg[0], cfg[1], cfg[2], K, bw, p64) for cfg in SWEEP}
    ms_step = max_over_ranks(total_ms / args.steps, dev)
    value = 100.0 * sum(ideal.values()) / (ms_step * 1e-3)

    sweep = []
    for cfg in SWEEP:
        flops, nbytes = model(cfg[0], cfg[1], cfg[2], K)
        ms = per_cfg[cfg]
        bound = "fp64" if flops / (p64 * 1e9) >= nbytes / (bw * 1e9) else "hbm"
        sweep.append({"dtype": "c64" if cfg[0] else "r64", "M": cfg[1], "N": cfg[2], "ms": round(ms, 4),
                      "gflops": round(flops / (ms * 1e-3) / 1e9, 2), "gbs": round(nbytes / (ms * 1e-3) / 1e9, 1),
                      "roofline_pct": round(100.0 * ideal[cfg] / (ms * 1e-3), 2), "bound": bound,
                      "variant": names[chosen[cfg][0]], "grid": chosen[cfg][1]})

    # our kernels per step: one per call, plus the final reduction pass of
    # the calls with many CTA partials
    lib = tsm.load()
    launches_per_step = sum(lib.tsm_tsmttsm_kernels_per_call(tsm.C64 if c[0] else tsm.R64, c[1], c[2],
                                                             chosen[c][1]) for c in SWEEP)

    # Dominant kernel: the longest call of the step.
    dom = max(SWEEP, key=lambda c: per_cfg[c])
    flops, nbytes = model(dom[0], dom[1], dom[2], K)
    dom_ms = per_cfg[dom]
    fp64_bound = flops / (p64 * 1e9) >= nbytes / (bw * 1e9)
    if fp64_bound:
        achieved = flops / (dom_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": p64 / 1e3, "unit": "TFLOP/s",
                "frac": achieved / (p64 / 1e3), "peak_source": "FP64 pipe, " + p64_src}
    else:
        achieved = nbytes / (dom_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": bw, "unit": "GB/s", "frac": achieved / bw,
                "peak_source": bw_src}
    cfg_key = "%s:%dx%d" % ("c64" if dom[0] else "r64", dom[1], dom[2])
    roof["traffic"] = _traffic_for(names[chosen[dom][0]], cfg_key)
    roof["kernel"] = names[chosen[dom][0]]
    roof["config"] = cfg_key

    # End to end: host (pinned) inputs copied in and C copied out every call.
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, flatA, flatB, outs, views, ideal, dev, K)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, wall = cpu_oracle_sweep(args.cpu_rows, K, bw, p64)
        cpu = {"value": v, "unit": "% of roofline", "cores": 1, "kind": "oracle",
               "sample": "first %d of 2^24 rows of each of the 22 sweep configurations (%.1f s of CPU), "
                         "times scaled x%d" % (args.cpu_rows, wall, K // args.cpu_rows)}

    extras = {}
    if rank == 0 and not args.no_extras:
        extras = run_extras(args, flatA, flatB, K, bw, p64)

    if rank == 0:
        line = {"metric": "TSMTTSM % of roofline vs width, K=2^24", "value": value, "unit": "% of roofline",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (SplitMix64 seeded, generated on device)",
                "config": {"workload": WORKLOAD, "K": K, "calls_per_step": len(SWEEP),
                           "l2": "inputs 2^24 rows >> 129 MB L2 except the C outputs; no flush",
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "gpu_launches": launches_per_step * args.steps,
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clock_info,
                "peaks": {"hbm_gbs": bw, "hbm_source": bw_src, "fp64_gflops_used": p64,
                          "fp64_source": p64_src, "fp64_nominal_gflops": FP64_NOMINAL_GFLOPS,
                          "dfma_probe_gflops": dfma, "dmma_probe_gflops": dmma},
                "sweep": sweep}
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_e2e(args, flatA, flatB, outs, views, ideal, dev, K):
    """One sweep where every call's A and B come from pinned host memory and
    the C results go back to the host: the same metric measured end to end.
    Each configuration's inputs are copied in full (no reuse across calls);
    the copies of the next configurations overlap the current kernel through
    a second stream and four device slots, and the 22 small results are read
    back behind the last product (a read-back after every call, on the
    compute stream, stalled the pipeline: one sweep took 2.7 s instead of
    1.4 s)."""
    import torch
    try:
        hA = torch.empty(flatA.numel(), dtype=torch.float64, pin_memory=True)
        hB = torch.empty(flatB.numel(), dtype=torch.float64, pin_memory=True)
        pinned = True
    except Exception:
        hA = torch.empty(flatA.numel(), dtype=torch.float64)
        hB = torch.empty(flatB.numel(), dtype=torch.float64)
        pinned = False
    hA.copy_(flatA)
    hB.copy_(flatB)
    nslot = 4  # device slots: the copies may run three calls ahead of the products
    slots = [(torch.empty_like(flatA), torch.empty_like(flatB)) for _ in range(nslot)]
    hC = {cfg: torch.empty(outs[cfg].shape, dtype=outs[cfg].dtype, pin_memory=pinned) for cfg in SWEEP}
    import paper_1905_03136_gb300 as tsm
    compute = torch.cuda.current_stream()
    copier = torch.cuda.Stream()
    h2d = d2h = 0
    copied = [torch.cuda.Event() for _ in SWEEP]
    done = [torch.cuda.Event() for _ in SWEEP]
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(compute)
    copier.wait_event(t0)
    for i, cfg in enumerate(SWEEP):
        cplx, M, N = cfg
        c = 2 if cplx else 1
        na, nb = K * M * c, K * N * c
        dA, dB = slots[i % nslot]
        with torch.cuda.stream(copier):
            if i >= nslot:
                copier.wait_event(done[i - nslot])
            dA[:na].copy_(hA[:na], non_blocking=True)
            dB[:nb].copy_(hB[:nb], non_blocking=True)
            copied[i].record(copier)
        compute.wait_event(copied[i])
        A, B = _views(dA, dB, cplx, M, N, K)
        tsm.tsmttsm(A, B, outs[cfg], op="C" if cplx else "T")
        done[i].record(compute)
        h2d += 8 * (na + nb)
    # the step's results back to the host, behind the last product
    for cfg in SWEEP:
        hC[cfg].copy_(outs[cfg], non_blocking=True)
        d2h += outs[cfg].numel() * outs[cfg].element_size()
    t1.record(compute)
    torch.cuda.synchronize()
    secs = t0.elapsed_time(t1) * 1e-3
    # raw pinned host-to-device bandwidth of one large copy, for context
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(compute)
    slots[0][0].copy_(hA, non_blocking=True)
    e1.record(compute)
    torch.cuda.synchronize()
    h2d_gbs = 8.0 * hA.numel() / (e0.elapsed_time(e1) * 1e-3) / 1e9
    del slots, hA, hB
    torch.cuda.empty_cache()
    return {"value": 100.0 * sum(ideal.values()) / secs, "unit": "% of roofline", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": secs * 1e3, "pinned": pinned,
            "h2d_gbs_single_copy": round(h2d_gbs, 1),
            "note": "every call copies its own A and B (no reuse) on a copy stream running up to three calls "
                    "ahead of the products (four device slots); the C results are read back at the end of the step"}


# ------------------------------------------------------------------ extras

def _reps_for(t_ideal_s):
    """Timed calls per point: several for calls below a millisecond, so that
    the host's launch latency of the first one (the start event is recorded
    behind a single warm-up call) is spread over them; one above."""
    return 1 if t_ideal_s > 1e-3 else 8


def _time(fn, reps=3, warm=1):
    """Mean milliseconds of `reps` calls, timed with CUDA events.  The start
    event is recorded behind the warm-up calls (no synchronisation between),
    so the timed calls find the host ahead of the GPU and their launch
    latency is hidden, as in a stream of calls."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    for _ in range(max(warm, 1)):
        fn()
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


SPLIT_CASES = [(True, 32, 32), (True, 48, 48), (True, 64, 64), (False, 64, 64)]
TSMM_SWEEP = [(c, m, n) for c in (False, True) for (m, n) in [(w, w) for w in SQUARE] + [(4, 64), (64, 4)]]


def run_split_extra(flatA, flatB, K, bw):
    """Split-precision TSMTTSM on the split workload: time, speed-up over the
    plain FP64 path, HBM fraction, and its normwise difference from the FP64
    path's result (both on the GPU; the oracle pins both in the tests)."""
    import torch
    import paper_1905_03136_gb300 as tsm
    from paper_1905_03136_gb300 import split
    out = []
    for dist in ("uniform", "loguniform"):
        tsm.fill_random(flatA.view(K, 128), 0, dist)
        tsm.fill_random(flatB.view(K, 128), 1, dist)
        for (cplx, M, N) in SPLIT_CASES:
            A, B = _views(flatA, flatB, cplx, M, N, K)
            op = "C" if cplx else "T"
            C1 = torch.zeros((M, N), dtype=A.dtype, device=A.device)
            C2 = torch.zeros_like(C1)
            ms_s = _time(lambda: split.tsmttsm_split(A, B, C1, op=op))
            status = split.status()
            ms_d = _time(lambda: tsm.tsmttsm(A, B, C2, op=op), reps=1)
            rel = float(torch.linalg.norm(C1 - C2) / torch.linalg.norm(C2))
            c = 2 if cplx else 1
            nbytes = 8.0 * c * (M + N) * K
            out.append({"dist": dist, "dtype": "c64" if cplx else "r64", "M": M, "N": N,
                        "ms_split": round(ms_s, 3), "ms_fp64": round(ms_d, 3), "speedup": round(ms_d / ms_s, 2),
                        "split_gbs": round(nbytes / (ms_s * 1e-3) / 1e9, 1),
                        "hbm_frac": round(nbytes / (ms_s * 1e-3) / 1e9 / bw, 3),
                        "rel_diff_vs_fp64_path": rel, "status": status})
    tsm.fill_random(flatA.view(K, 128), 0)
    tsm.fill_random(flatB.view(K, 128), 1)
    return out


def run_tsmm_extra(flatA, flatB, K, bw, p64):
    import torch
    import paper_1905_03136_gb300 as tsm
    out, ideal, meas = [], 0.0, 0.0
    Bout = torch.empty(K * 128, dtype=torch.float64, device=flatA.device)
    for (cplx, M, N) in TSMM_SWEEP:
        c = 2 if cplx else 1
        A = flatA[: K * M * c]
        Cm = flatB[: M * N * c]
        Bo = Bout[: K * N * c]
        if cplx:
            A, Cm, Bo = A.view(torch.complex128), Cm.view(torch.complex128), Bo.view(torch.complex128)
        A, Cm, Bo = A.view(K, M), Cm.view(M, N), Bo.view(K, N)
        flops, nbytes = model(cplx, M, N, K)
        t_ideal = max(nbytes / (bw * 1e9), flops / (p64 * 1e9))
        ms = _time(lambda: tsm.tsmm(A, Cm, Bo), reps=_reps_for(t_ideal))
        ideal += t_ideal
        meas += ms * 1e-3
        out.append({"dtype": "c64" if cplx else "r64", "M": M, "N": N, "ms": round(ms, 4),
                    "roofline_pct": round(100 * t_ideal / (ms * 1e-3), 2)})
    del Bout
    torch.cuda.empty_cache()
    return {"roofline_pct_whole_sweep": 100 * ideal / meas, "calls": out}


def run_widths_extra(flatA, flatB, K, bw, p64):
    """Every width: M = N = w for w = 1..64 at K = 2^24, real and complex,
    TSMTTSM (op T real, op C complex) and TSMM with beta = 0 and beta = 1
    (beta = 1 also reads B: 8cNK more bytes).  One warm-up call and one to
    eight timed calls per point; percent of roofline per width and the
    widths below 90 %."""
    import torch
    import paper_1905_03136_gb300 as tsm
    Bout = torch.empty(K * 128, dtype=torch.float64, device=flatA.device)
    Bout.zero_()
    res = {}
    below = []
    for kind in ("tsmttsm", "tsmm_beta0", "tsmm_beta1"):
        res[kind] = {}
        for cplx in (False, True):
            c = 2 if cplx else 1
            dt = torch.complex128 if cplx else torch.float64
            pct, ms_list = [], []
            for w in range(1, 65):
                A = flatA[: K * w * c]
                if cplx:
                    A = A.view(torch.complex128)
                A = A.view(K, w)
                flops, nbytes = model(cplx, w, w, K)
                if kind == "tsmm_beta1":
                    nbytes += 8.0 * c * w * K
                t_ideal = max(nbytes / (bw * 1e9), flops / (p64 * 1e9))
                reps = _reps_for(t_ideal)
                if kind == "tsmttsm":
                    Bm = flatB[: K * w * c]
                    Bm = (Bm.view(torch.complex128) if cplx else Bm).view(K, w)
                    C = torch.zeros((w, w), dtype=dt, device=flatA.device)
                    ms = _time(lambda: tsm.tsmttsm(A, Bm, C, op="C" if cplx else "T"), reps=reps)
                else:
                    beta = 0.0 if kind == "tsmm_beta0" else 1.0
                    Cm = flatB[: w * w * c]
                    Cm = (Cm.view(torch.complex128) if cplx else Cm).view(w, w)
                    Bo = Bout[: K * w * c]
                    Bo = (Bo.view(torch.complex128) if cplx else Bo).view(K, w)
                    ms = _time(lambda: tsm.tsmm(A, Cm, Bo, 1.0, beta), reps=reps)
                p = 100.0 * t_ideal / (ms * 1e-3)
                pct.append(round(p, 1))
                ms_list.append(round(ms, 4))
                if p < 90.0:
                    below.append("%s %s w=%d: %.1f" % (kind, "c64" if cplx else "r64", w, p))
            res[kind]["c64" if cplx else "r64"] = {"roofline_pct": pct, "ms": ms_list,
                                                   "min_pct": min(pct), "min_at_w": 1 + pct.index(min(pct))}
    del Bout
    torch.cuda.empty_cache()
    res["what"] = ("M = N = w for w = 1..64 at K = 2^24: percent of roofline per width (index w - 1), "
                   "TSMTTSM and TSMM (beta 0 / 1), real and complex")
    res["below_90"] = below
    return res


GS_CASES = [(True, 32, 32), (True, 64, 64), (False, 64, 64), (False, 8, 8)]


def run_gs_extra(flatA, flatB, K, bw, p64):
    """Block Gram-Schmidt step (C = A^H B, B -= A C) through tsm_gs_step at
    K = 2^24: time against the sum of the two products' roofline times (the
    TSMM reads and writes B: beta = 1)."""
    import torch
    import paper_1905_03136_gb300 as tsm
    out, ideal, meas = [], 0.0, 0.0
    Bw = torch.empty(K * 128, dtype=torch.float64, device=flatA.device)
    for (cplx, M, N) in GS_CASES:
        c = 2 if cplx else 1
        A = flatA[: K * M * c]
        B = Bw[: K * N * c]
        B.copy_(flatB[: K * N * c])
        if cplx:
            A, B = A.view(torch.complex128), B.view(torch.complex128)
        A, B = A.view(K, M), B.view(K, N)
        C = torch.empty((M, N), dtype=A.dtype, device=A.device)
        ms = _time(lambda: tsm.gs_step(A, B, C), reps=2)
        f1, b1 = model(cplx, M, N, K)
        b2 = b1 + 8.0 * c * N * K  # TSMM with beta = 1 also reads B
        t_ideal = max(b1 / (bw * 1e9), f1 / (p64 * 1e9)) + max(b2 / (bw * 1e9), f1 / (p64 * 1e9))
        ideal += t_ideal
        meas += ms * 1e-3
        out.append({"dtype": "c64" if cplx else "r64", "M": M, "N": N, "ms": round(ms, 4),
                    "roofline_pct": round(100 * t_ideal / (ms * 1e-3), 2)})
    del Bw
    torch.cuda.empty_cache()
    return {"what": "tsm_gs_step: TSMTTSM (op C) then TSMM (alpha=-1, beta=1) on one stream, C on the device",
            "roofline_pct_all": 100 * ideal / meas, "calls": out}


RAMP_K = [10 ** 4, 3 * 10 ** 4, 10 ** 5, 3 * 10 ** 5, 10 ** 6, 1 << 21, 1 << 22, 1 << 24]
RAMP_CASES = [(False, 4, 4), (False, 16, 16), (True, 8, 8), (True, 32, 32)]


def run_ramp_extra(flatA, flatB, bw, p64):
    """Small-K ramp (the paper's Fig. 18 experiment): percent of roofline of
    the tuned TSMTTSM as K grows from 10^4 to 2^24.  `fixed_us` is the time
    of a call with one 16-row slab per CTA (K = 16 x grid): launch, the
    in-CTA and the cross-CTA reductions, and the epilogue, with almost no
    streaming; `fixed_share` is that time over each call's time.  Calls are
    timed back to back through the library's own timer (tsm_time_variant,
    one warm-up call, then CUDA events around the repetitions), so that a
    call of a few microseconds is not hidden behind Python's launch cost."""
    import torch
    import paper_1905_03136_gb300 as tsm
    res = []
    for (cplx, M, N) in RAMP_CASES:
        dt = tsm.C64 if cplx else tsm.R64
        C = torch.zeros((M, N), dtype=torch.complex128 if cplx else torch.float64, device=flatA.device)
        var, grid = tsm.choose(tsm.KIND_TSMTTSM, dt, M, N, 1 << 20)
        k0 = 16 * max(grid, 1)
        A0, B0 = _views(flatA, flatB, cplx, M, N, k0)
        fixed = tsm.time_variant(tsm.KIND_TSMTTSM, A0, B0, C, var, grid, reps=50)
        pts = []
        for K in RAMP_K:
            A, B = _views(flatA, flatB, cplx, M, N, K)
            v, g = tsm.choose(tsm.KIND_TSMTTSM, dt, M, N, K)
            reps = 50 if K <= (1 << 22) else 3
            ms = tsm.time_variant(tsm.KIND_TSMTTSM, A, B, C, v, g, reps=reps)
            t_ideal = ideal_seconds(cplx, M, N, K, bw, p64)
            pts.append({"K": K, "us": round(ms * 1e3, 2), "roofline_pct": round(100 * t_ideal / (ms * 1e-3), 2),
                        "fixed_share": round(fixed / ms, 4)})
        res.append({"dtype": "c64" if cplx else "r64", "M": M, "N": N, "grid_at_2^20": grid,
                    "fixed_us": round(fixed * 1e3, 2), "points": pts})
    return {"what": "TSMTTSM % of roofline vs K (tuned variant per K)", "cases": res}


def batched_workload(seed=0, count=256):
    """The batched mixed workload: op TSMTTSM/TSMM and dtype 50/50, M, N
    uniform in [1, 64], K = floor(2^(16 + 6u)) (log-uniform in [2^16, 2^22])."""
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        out.append((int(rng.integers(0, 2)), bool(rng.integers(0, 2)), int(rng.integers(1, 65)),
                    int(rng.integers(1, 65)), int(2 ** (16 + 6 * rng.random()))))
    return out


def batched_configs_from_model(insts, model):
    """Per-instance configuration picked by the cost model among the batched
    kernel's codes (tile codes for TSMTTSM, threads-per-row codes for TSMM)."""
    import numpy as np
    from paper_1905_03136_gb300 import costmodel as cm
    import paper_1905_03136_gb300 as tsm
    tiles = {1: (1, 1, 4), 2: (2, 2, 2), 3: (4, 4, 1), 4: (4, 8, 1), 5: (8, 4, 1), 6: (3, 3, 2), 7: (2, 5, 2),
             8: (5, 2, 2), 9: (3, 5, 1), 10: (5, 3, 1), 11: (2, 7, 1), 12: (7, 2, 1)}
    tprs = {1: 4, 2: 8, 3: 16}
    rt = {v["dtype"]: v["index"] for v in tsm.variants(tsm.KIND_TSMM) if v["name"].endswith("_rt_npt4_u2")}
    cfg = []
    for (kind, cplx, M, N, K) in insts:
        cands, feats = [], []
        if kind == 0:
            for code, (tm, tn, u) in tiles.items():
                if cplx and code in (4, 5):
                    tm, tn = 4, 4  # complex runs these codes with a 4x4 tile
                if math.ceil(M / tm) * math.ceil(N / tn) > 256:
                    continue
                cands.append(code)
                feats.append(cm.featurize(0, int(cplx), M, N, K, tm, tn, 1, u, 0, 0, 152))
        else:
            for code, tpr in tprs.items():
                if cplx and code == 1:
                    tpr = 8
                cands.append(code)
                feats.append(cm.featurize(1, int(cplx), M, N, K, 1, math.ceil(N / tpr), tpr, 2, 0, 0, 152))
            shape = tsm.variant_shape(tsm.KIND_TSMM, rt[int(cplx)], int(cplx), M, N)
            cands.append(4)
            feats.append(cm.featurize(1, int(cplx), M, N, K, 1, shape["tile_n"], shape["threads_per_row"], 2, 0, 0,
                                      152))
        pred = model.predict_log2_ineff(feats)
        cfg.append(cands[int(np.argmin(pred))])
    return cfg


def run_batched_extra(flatA, flatB):
    """256 instances in one graph launch: default configurations vs the cost
    model's, against launching every instance separately."""
    import torch
    from paper_1905_03136_gb300 import batched as bt
    from paper_1905_03136_gb300 import costmodel as cm
    import paper_1905_03136_gb300 as tsm
    insts = batched_workload()
    dev = flatA.device
    outs, views = [], []
    for (kind, cplx, M, N, K) in insts:
        c = 2 if cplx else 1
        dt = torch.complex128 if cplx else torch.float64
        A = flatA[: K * M * c]
        if kind == 0:
            B = flatB[: K * N * c]
            O = torch.zeros(M * N * c, dtype=torch.float64, device=dev)
        else:
            B = flatB[: M * N * c]
            O = torch.zeros(K * N * c, dtype=torch.float64, device=dev)
        if cplx:
            A, B, O = A.view(dt), B.view(dt), O.view(dt)
        A = A.view(K, M)
        B = B.view(K, N) if kind == 0 else B.view(M, N)
        O = O.view(M, N) if kind == 0 else O.view(K, N)
        views.append((A, B, O))
    flops = sum(2.0 * M * N * K * (4 if c else 1) for (_, c, M, N, K) in insts)
    res = {"instances": len(insts), "flops": flops}

    def make(cfgs):
        descs = [bt.desc(k, A, B, O, 1.0, 0.0, ("C" if c else "T") if k == 0 else "N", cfg)
                 for (k, c, M, N, K), (A, B, O), cfg in zip(insts, views, cfgs)]
        return bt.Batch(descs)

    default = make([0] * len(insts))
    res["items"], res["ctas"] = default.info()
    res["default_graph_ms"] = _time(default.run, reps=2)
    res["default_direct_ms"] = _time(default.run_direct, reps=1)
    default.close()
    model_path = os.path.join(ROOT, "paper_1905_03136_gb300", "tuning", "costmodel.npz")
    if os.path.exists(model_path):
        model = cm.CostModel()
        model.load(model_path)
        b = make(batched_configs_from_model(insts, model))
        res["mlp_graph_ms"] = _time(b.run, reps=2)
        b.close()

    def separate():
        for (k, c, M, N, K), (A, B, O) in zip(insts, views):
            if k == 0:
                tsm.tsmttsm(A, B, O, op="C" if c else "T")
            else:
                tsm.tsmm(A, B, O)
    res["separate_launches_ms"] = _time(separate, reps=1)
    res["gflops_default_graph"] = flops / (res["default_graph_ms"] * 1e-3) / 1e9
    del views, outs
    torch.cuda.empty_cache()
    return res


def run_cublas_extra(flatA, flatB, K, bw, p64):
    """The same sweep through cuBLAS (torch.matmul on transposed views of the
    same buffers: DGEMM with op T, ZGEMM with op C), for comparison with the
    library's kernels; percent of the same roofline."""
    import torch
    rows = []
    ideal_sum = meas_sum = 0.0
    for cfg in SWEEP:
        A, B = _views(flatA, flatB, cfg[0], cfg[1], cfg[2], K)
        At = A.mH if cfg[0] else A.t()
        out = torch.matmul(At, B)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        e0.record()
        for _ in range(reps):
            out = torch.matmul(At, B)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        ideal = ideal_seconds(cfg[0], cfg[1], cfg[2], K, bw, p64)
        ideal_sum += ideal
        meas_sum += ms * 1e-3
        rows.append({"dtype": "c64" if cfg[0] else "r64", "M": cfg[1], "N": cfg[2], "ms": round(ms, 4),
                     "roofline_pct": round(100.0 * ideal / (ms * 1e-3), 2)})
        del out
    return {"what": "cuBLAS DGEMM (op T) / ZGEMM (op C) via torch.matmul on the same buffers",
            "value": 100.0 * ideal_sum / meas_sum, "unit": "% of roofline", "sweep": rows}


def run_extras(args, flatA, flatB, K, bw, p64):
    ex = {}
    try:
        ex["cublas"] = run_cublas_extra(flatA, flatB, K, bw, p64)
    except Exception as e:  # reported, never hidden
        ex["cublas"] = {"error": repr(e)}
    try:
        ex["split"] = run_split_extra(flatA, flatB, K, bw)
    except Exception as e:  # reported, never hidden
        ex["split"] = {"error": repr(e)}
    try:
        ex["tsmm_sweep"] = run_tsmm_extra(flatA, flatB, K, bw, p64)
    except Exception as e:
        ex["tsmm_sweep"] = {"error": repr(e)}
    try:
        ex["widths"] = run_widths_extra(flatA, flatB, K, bw, p64)
    except Exception as e:
        ex["widths"] = {"error": repr(e)}
    try:
        ex["gs_step"] = run_gs_extra(flatA, flatB, K, bw, p64)
    except Exception as e:
        ex["gs_step"] = {"error": repr(e)}
    try:
        ex["small_k_ramp"] = run_ramp_extra(flatA, flatB, bw, p64)
    except Exception as e:
        ex["small_k_ramp"] = {"error": repr(e)}
    try:
        ex["batched"] = run_batched_extra(flatA, flatB)
    except Exception as e:
        ex["batched"] = {"error": repr(e)}
    return ex


def main():
    ap = argparse.ArgumentParser(description="TSMTTSM roofline sweep benchmark")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--cpu-rows", type=int, default=1 << 17, help="rows of the CPU-oracle sample per config")
    ap.add_argument("--ref-rows", type=int, default=1 << 14, help="rows per config per reference-arm step")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the split / TSMM / batched extras")
    ap.add_argument("--case", default=None, help="profile one config, e.g. c64:64x64")
    ap.add_argument("--k", type=int, default=1 << 20, help="rows for --case")
    ap.add_argument("--split", action="store_true", help="--case: use the split-precision path")
    args = ap.parse_args()
    bw, bw_src = load_peaks()
    if args.case:
        return run_case(args)
    if args.impl == "reference":
        if int(os.environ.get("RANK", "0")) != 0:
            return
        return run_reference(args, bw, bw_src)
    return run_ours(args, bw, bw_src)


if __name__ == "__main__":
    main()
