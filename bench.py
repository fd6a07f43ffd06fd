#!/usr/bin/env python
"""Benchmark: TSMTTSM / TSMM percent of roofline over the width sweeps at K = 2^24.

One step = one pass of both products over the width sweeps, on inputs
already resident in HBM (58 kernel calls):
  * TSMTTSM (real op T, complex op C; alpha = 1, beta = 0) for
    M = N in {1, 2, 4, 8, 16, 32, 64} and (M, N) in {(1,64), (64,1), (8,32),
    (32,8)};
  * TSMM (alpha = 1, beta = 0 and beta = 1) for M = N in {1, ..., 64 by
    powers of two} and (M, N) in {(4,64), (64,4)}.

Roofline per call (Sec. 1.3, Eq. 1): flops = 2MNK (real) or 8MNK (complex),
bytes = 8c(MK + NK + MN) (c = 2 for complex; TSMM with beta != 0 also reads
B: + 8cNK), P_max = min(I * b_s, P_fp64) with b_s the measured HBM copy
bandwidth (MEASURED_PEAKS.json) and P_fp64 the FP64 rate measured live by
the library's DFMA probe.  The reported value is whole-step efficiency:
100 * sum(ideal time) / step time.

Output: every extra measurement (per-width sweep, split path, small-K ramp,
batched launch, cuBLAS, ...) is printed on a JSON line of its own
({"extra": name, ...}) and, with --extras-out, written to one JSON file;
the LAST stdout line is the compact headline record.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       python bench.py --case c64:64x64 --k 1048576   (one kernel, for profiling)
"""

import argparse
import hashlib
import json
import math
import os
import platform
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
TSMM_SWEEP = [(c, m, n) for c in (False, True) for (m, n) in [(w, w) for w in SQUARE] + [(4, 64), (64, 4)]]
# the calls of one step: (kind, complex, M, N, beta)
STEP = [("tsmttsm", c, m, n, 0.0) for (c, m, n) in SWEEP] + \
       [("tsmm", c, m, n, b) for (c, m, n) in TSMM_SWEEP for b in (0.0, 1.0)]
FP64_NOMINAL_GFLOPS = 1250.0   # GB300 FP64 (vector and tensor), per GPU, for context only
HBM_FALLBACK_GBS = 6800.0
METRIC = "TSMTTSM/TSMM % of roofline (HBM GB/s or FP64 TF/s) vs width 1–64, K=2^24"
WORKLOAD = ("FP64 width sweeps at K=2^24, row-major, ld=width, uniform(-1,1) SplitMix64 inputs (A seed 0, "
            "B seed 1, C seed 2): TSMTTSM real op T + complex op C, M=N in {1,2,4,...,64} + (M,N) in "
            "{(1,64),(64,1),(8,32),(32,8)}, alpha=1, beta=0; TSMM real + complex, M=N in {1,2,4,...,64} + "
            "(4,64),(64,4), alpha=1, beta in {0,1}")


def model(cplx, M, N, K):
    """(flops, bytes) of one TSMTTSM call with beta = 0 (Eq. 1 of the paper,
    complex: 4x flops, 2x bytes)."""
    c = 2 if cplx else 1
    flops = 2.0 * M * N * K * (4 if cplx else 1)
    nbytes = 8.0 * c * (M * K + N * K + M * N)
    return flops, nbytes


def call_model(kind, cplx, M, N, K, beta):
    """(flops, bytes) of one call: Eq. 1, plus the read of B for a TSMM with
    beta != 0 (and of C for a TSMTTSM with beta != 0)."""
    flops, nbytes = model(cplx, M, N, K)
    c = 2 if cplx else 1
    if beta != 0.0:
        nbytes += 8.0 * c * (N * K if kind == "tsmm" else M * N)
    return flops, nbytes


def ideal_seconds(cplx, M, N, K, bw_gbs, p64_gflops, kind="tsmttsm", beta=0.0):
    flops, nbytes = call_model(kind, cplx, M, N, K, beta)
    return max(nbytes / (bw_gbs * 1e9), flops / (p64_gflops * 1e9))


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


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
    FP64 family, the narrow kernels or the generator, plus their shared
    epilogue and header."""
    h = hashlib.sha256()
    pkg = os.path.join(ROOT, "paper_1905_03136_gb300")
    files = ["csrc/fp64_common.cuh", "csrc/tsm_internal.h"]
    if variant_name.startswith("gen_"):
        files.append("codegen.py")
    elif "narrow" in variant_name:
        files.append("csrc/kernels_narrow.cu")
    elif "_rt_" in variant_name:
        files.append("csrc/kernels_rt.cu")
    else:
        files += ["csrc/kernels_fp64.cu", "csrc/fp64_tsmttsm.cuh"]
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


def _mat(flat, rows, cols, cplx):
    """A (rows x cols) row-major view of the start of a flat float64 buffer."""
    import torch
    v = flat[: rows * cols * (2 if cplx else 1)]
    if cplx:
        v = v.view(torch.complex128)
    return v.view(rows, cols)


# ------------------------------------------------------------------ CPU baseline

def _host_flat(seed, rows):
    """Flat host buffer of rows x 128 doubles: by the element addressing of
    ``synth`` its first K*w(*2) doubles are the seeded input of every width
    w (and of every complex width) with ld = w."""
    import synth
    return synth.block_vector(seed, rows, 128).reshape(-1)


def cpu_step(hA, hB, hC, hO, K, threads):
    """Seconds of one step of the plain CPU loops on the first K rows of every
    call of the step (input generation outside the timed region)."""
    import numpy as np
    import oracle
    secs = []
    for (kind, cplx, M, N, beta) in STEP:
        dt = np.complex128 if cplx else np.float64
        c = 2 if cplx else 1
        A = hA[: K * M * c].view(dt)
        if kind == "tsmttsm":
            B = hB[: K * N * c].view(dt)
            C = np.zeros(M * N, dtype=dt)
            t0 = time.perf_counter()
            oracle.tsmttsm_plain("C" if cplx else "T", M, N, K, 1.0, A, M, B, N, 0.0, C, N, threads)
        else:
            Cm = hC[: M * N * c].view(dt)
            O = hO[: K * N * c].view(dt)
            t0 = time.perf_counter()
            oracle.tsmm_plain(M, N, K, 1.0, A, M, Cm, N, beta, O, N, threads)
        secs.append(time.perf_counter() - t0)
    return secs


def cpu_baseline(K_single, K_all, bw, p64):
    """The plain CPU loops (oracle/tsm_plain.c, as they stand) on one host
    core and on every host core, each on the first rows of every call of
    the step, times scaled linearly to K = 2^24 (every call's work grows
    linearly in K).  Returns the cpu_baseline record."""
    import numpy as np
    Kmax = max(K_single, K_all)
    hA, hB = _host_flat(0, Kmax), _host_flat(1, Kmax)
    hC = _host_flat(2, 64)
    hO = np.zeros(Kmax * 128)
    ideal = sum(ideal_seconds(c, M, N, K_FULL, bw, p64, kind, b) for (kind, c, M, N, b) in STEP)
    cores = host_cores()
    out = {}
    for label, K, T in (("single", K_single, 1), ("all", K_all, cores)):
        secs = cpu_step(hA, hB, hC, hO, K, T)
        out[label] = (100.0 * ideal / (sum(secs) * K_FULL / K), sum(secs))
    return {"value": out["all"][0], "unit": "% of roofline", "cores": cores, "kind": "oracle",
            "sample": "plain uncompensated loops of oracle/tsm_plain.c: first %d rows of each of the %d calls "
                      "on %d threads (%.1f s), first %d rows on 1 thread (%.1f s); times scaled to 2^24 rows"
                      % (K_all, len(STEP), cores, out["all"][1], K_single, out["single"][1]),
            "single_core_value": out["single"][0], "cpu": cpu_model()}


# ------------------------------------------------------------------ arms

def run_reference(args, bw, bw_src):
    """The reference arm: the plain CPU loops on every host core, each step a
    bounded sample (the first --ref-rows rows of every call of the step,
    times scaled linearly to 2^24 rows)."""
    import numpy as np
    p64 = FP64_NOMINAL_GFLOPS
    K_s = args.ref_rows
    hA, hB, hC = _host_flat(0, K_s), _host_flat(1, K_s), _host_flat(2, 64)
    hO = np.zeros(K_s * 128)
    cores = host_cores()
    ideal = sum(ideal_seconds(c, M, N, K_FULL, bw, p64, kind, b) for (kind, c, M, N, b) in STEP)
    for _ in range(args.warmup):
        cpu_step(hA, hB, hC, hO, K_s, cores)
    walls = []
    for _ in range(args.steps):
        walls.append(sum(cpu_step(hA, hB, hC, hO, K_s, cores)))
    secs = statistics.mean(walls)
    value = 100.0 * ideal / (secs * K_FULL / K_s)
    sample = ("plain uncompensated loops of oracle/tsm_plain.c on %d threads: first %d of 2^24 rows of each of "
              "the %d calls of the step, times scaled x%d" % (cores, K_s, len(STEP), K_FULL // K_s))
    line = {"impl": "reference", "metric": METRIC, "value": value,
            "unit": "% of roofline", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (SplitMix64 seeded)",
            "config": {"workload": WORKLOAD, "K": K_FULL, "parallelism": "replicas"},
            "cpu_baseline": {"value": value, "unit": "% of roofline", "cores": cores, "kind": "oracle",
                             "sample": sample, "cpu": cpu_model()},
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
    fb = torch.empty(K * max(M, N) * c, dtype=torch.float64, device="cuda")
    tsm.fill_random(fa.view(1, -1), 0)
    tsm.fill_random(fb.view(1, -1), 1)
    if args.tsmm:
        A = _mat(fa, K, M, cplx)
        Cm = _mat(fb, M, N, cplx).clone()
        Bo = _mat(fb, K, N, cplx)
        for _ in range(args.steps):
            tsm.tsmm(A, Cm, Bo, 1.0, args.beta)
    else:
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


def measure_fp64_peak(local):
    """The FP64 rate of the library's probes (DFMA register tile, FP64 MMA,
    constant-operand DFMA chain), with the SM clock sampled while they run.
    The register-tile DFMA form is the one the products use."""
    from paper_1905_03136_gb300 import probe
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.2)
    dfma = probe.fp64_peak(0, iters=30000)
    dmma = probe.fp64_peak(1, iters=20000)
    chain = probe.fp64_peak(2, iters=40000)
    info = clocks.stop()
    return {"dfma_tile": dfma, "dmma": dmma, "dfma_chain": chain, "sm_mhz": info.get("sm_mhz"),
            "reasons": info.get("reasons")}


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
    lib = tsm.load()
    dev = torch.device("cuda", local)
    K = K_FULL
    extras_file = {}

    def emit(name, rec):
        """An extra measurement: its own stdout line now, the file later."""
        extras_file[name] = rec
        if rank == 0:
            print(json.dumps({"extra": name, **(rec if isinstance(rec, dict) else {"value": rec})}), flush=True)

    # Inputs: one flat buffer per operand, seeded once (outside timing).  By
    # the generator's element addressing the prefix of K*w(*2) doubles is the
    # seeded input of every width w with ld = w (see _host_flat).
    flatA = torch.empty(K * 128, dtype=torch.float64, device=dev)
    flatB = torch.empty(K * 128, dtype=torch.float64, device=dev)
    flatC = torch.empty(64 * 128, dtype=torch.float64, device=dev)
    Bout = torch.zeros(K * 128, dtype=torch.float64, device=dev)
    tsm.fill_random(flatA.view(K, 128), 0)
    tsm.fill_random(flatB.view(K, 128), 1)
    tsm.fill_random(flatC.view(64, 128), 2)
    kdt = {False: tsm.R64, True: tsm.C64}

    calls = []
    for (kind, cplx, M, N, beta) in STEP:
        A = _mat(flatA, K, M, cplx)
        if kind == "tsmttsm":
            B = _mat(flatB, K, N, cplx)
            out = torch.zeros((M, N), dtype=A.dtype, device=dev)
            var, grid = tsm.choose(tsm.KIND_TSMTTSM, kdt[cplx], M, N, K)
            fn = (lambda A=A, B=B, out=out, op=("C" if cplx else "T"): tsm.tsmttsm(A, B, out, op=op))
            launches = lib.tsm_tsmttsm_kernels_per_call(kdt[cplx], M, N, grid)
        else:
            Cm = _mat(flatC, M, N, cplx)
            out = _mat(Bout, K, N, cplx)
            var, grid = tsm.choose(tsm.KIND_TSMM_BETA if beta else tsm.KIND_TSMM, kdt[cplx], M, N, K)
            fn = (lambda A=A, Cm=Cm, out=out, beta=beta: tsm.tsmm(A, Cm, out, 1.0, beta))
            launches = 1
        calls.append({"key": (kind, cplx, M, N, beta), "fn": fn, "var": var, "grid": grid, "launches": launches})
    names = {k: {v["index"]: v["name"] for v in tsm.variants(k)} for k in (tsm.KIND_TSMTTSM, tsm.KIND_TSMM)}

    fp64 = measure_fp64_peak(local)
    p64 = max(fp64["dfma_tile"], fp64["dmma"], fp64["dfma_chain"])
    p64_src = "measured: DFMA register-tile probe at %s MHz" % fp64["sm_mhz"] if p64 == fp64["dfma_tile"] else \
        "measured: %s probe" % ("FP64 MMA" if p64 == fp64["dmma"] else "DFMA chain")

    stream = torch.cuda.current_stream()

    def step(record=None):
        for i, cl in enumerate(calls):
            if record is not None:
                record[i][0].record(stream)
            cl["fn"]()
            if record is not None:
                record[i][1].record(stream)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()

    events = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in calls]
              for _ in range(args.steps)]
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
    # latency (the whole-step value keeps it).
    per_call = [statistics.median(events[s][i][0].elapsed_time(events[s][i][1]) for s in range(args.steps))
                for i in range(len(calls))]

    ideal = [ideal_seconds(cplx, M, N, K, bw, p64, kind, beta) for (kind, cplx, M, N, beta) in STEP]
    ms_step = max_over_ranks(total_ms / args.steps, dev)
    value = 100.0 * sum(ideal) / (ms_step * 1e-3)

    rows = []
    for i, cl in enumerate(calls):
        kind, cplx, M, N, beta = cl["key"]
        flops, nbytes = call_model(kind, cplx, M, N, K, beta)
        ms = per_call[i]
        nm = names[tsm.KIND_TSMTTSM if kind == "tsmttsm" else tsm.KIND_TSMM][cl["var"]]
        rows.append({"kind": kind, "dtype": "c64" if cplx else "r64", "M": M, "N": N, "beta": beta,
                     "ms": round(ms, 4), "gflops": round(flops / (ms * 1e-3) / 1e9, 2),
                     "gbs": round(nbytes / (ms * 1e-3) / 1e9, 1),
                     "roofline_pct": round(100.0 * ideal[i] / (ms * 1e-3), 2),
                     "bound": "fp64" if flops / (p64 * 1e9) >= nbytes / (bw * 1e9) else "hbm",
                     "variant": nm, "grid": cl["grid"]})
    emit("step_calls", {"calls": rows})
    part = {}
    for kind in ("tsmttsm", "tsmm"):
        idx = [i for i, cl in enumerate(calls) if cl["key"][0] == kind]
        part[kind] = round(100.0 * sum(ideal[i] for i in idx) / (1e-3 * sum(per_call[i] for i in idx)), 2)

    launches_per_step = sum(cl["launches"] for cl in calls)

    # Dominant kernel: the longest call of the step.
    d = max(range(len(calls)), key=lambda i: per_call[i])
    kind, cplx, M, N, beta = calls[d]["key"]
    flops, nbytes = call_model(kind, cplx, M, N, K, beta)
    dom_ms = per_call[d]
    dom_name = names[tsm.KIND_TSMTTSM if kind == "tsmttsm" else tsm.KIND_TSMM][calls[d]["var"]]
    if flops / (p64 * 1e9) >= nbytes / (bw * 1e9):
        achieved = flops / (dom_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": round(achieved, 4), "peak": round(p64 / 1e3, 4), "unit": "TFLOP/s",
                "frac": round(achieved / (p64 / 1e3), 4), "peak_source": "FP64 pipe, " + p64_src}
    else:
        achieved = nbytes / (dom_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": bw, "unit": "GB/s",
                "frac": round(achieved / bw, 4), "peak_source": bw_src}
    cfg_key = "%s:%s:%dx%d%s" % (kind, "c64" if cplx else "r64", M, N, ":beta1" if beta else "")
    roof["traffic"] = _traffic_for(dom_name, cfg_key)
    roof["kernel"] = dom_name
    roof["config"] = cfg_key
    roof["ms"] = round(dom_ms, 3)

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(calls, flatA, flatB, flatC, sum(ideal), dev, K)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(args.cpu_rows, args.cpu_rows_all, bw, p64)

    summary = {}
    if rank == 0 and not args.no_extras:
        summary = run_extras(args, flatA, flatB, K, bw, p64, emit)

    if rank == 0:
        emit("peaks", {"hbm_gbs": bw, "hbm_source": bw_src, "fp64_gflops_used": p64, "fp64_source": p64_src,
                       "fp64_nominal_gflops": FP64_NOMINAL_GFLOPS, "probes": fp64})
        if args.extras_out:
            with open(args.extras_out, "w") as f:
                json.dump(extras_file, f)
        line = {"metric": METRIC, "value": round(value, 3), "unit": "% of roofline",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (SplitMix64 seeded, generated on device)",
                "config": {"workload": "TSMTTSM 22-call + TSMM 36-call FP64 width sweeps, K=2^24 (A seed 0, "
                                       "B seed 1, C seed 2, uniform(-1,1))", "K": K, "calls_per_step": len(calls),
                           "l2": "inputs 2^24 rows >> 129 MB L2; no flush",
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "gpu_launches": launches_per_step * args.steps,
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": {k: clock_info.get(k) for k in ("sm_mhz", "sm_max_mhz", "reasons", "power_w_max")},
                "fp64_peak_gflops": round(p64, 1),
                "by_product_pct": part}
        line.update(summary)
        text = json.dumps(line)
        if len(text) > 2600:  # the headline must stay short: drop the extras summary first
            for k in list(summary):
                line.pop(k, None)
            text = json.dumps(line)
        print(text, flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_e2e(calls, flatA, flatB, flatC, ideal_s, dev, K):
    """One step of the same 58 calls through the public API with host
    inputs: every call's A, B and C come from pinned host memory and every
    result goes back to pinned host memory, copies inside the timed region.
    Copies of the next calls run on a copy-in stream up to two calls ahead
    of the products (three device slots); TSMM results go back on a
    copy-out stream as soon as their kernel ends; the 22 small TSMTTSM
    results are read back behind the last product."""
    import torch
    import paper_1905_03136_gb300 as tsm
    try:
        hA = torch.empty(flatA.numel(), dtype=torch.float64, pin_memory=True)
        hB = torch.empty(flatB.numel(), dtype=torch.float64, pin_memory=True)
        hO = torch.empty(flatB.numel(), dtype=torch.float64, pin_memory=True)
        pinned = True
    except Exception:
        hA = torch.empty(flatA.numel(), dtype=torch.float64)
        hB = torch.empty(flatB.numel(), dtype=torch.float64)
        hO = torch.empty(flatB.numel(), dtype=torch.float64)
        pinned = False
    hA.copy_(flatA)
    hB.copy_(flatB)
    hCin = flatC.cpu()
    nslot = 3
    slots = [(torch.empty_like(flatA), torch.empty_like(flatB), torch.empty_like(flatC)) for _ in range(nslot)]
    small_out = []
    compute = torch.cuda.current_stream()
    cin, cout = torch.cuda.Stream(), torch.cuda.Stream()
    n = len(calls)
    copied = [torch.cuda.Event() for _ in range(n)]
    done = [torch.cuda.Event() for _ in range(n)]
    freed = [torch.cuda.Event() for _ in range(n)]
    h2d = d2h = 0
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(compute)
    cin.wait_event(t0)
    for i, cl in enumerate(calls):
        kind, cplx, M, N, beta = cl["key"]
        c = 2 if cplx else 1
        dA, dB, dC = slots[i % nslot]
        na, nb = K * M * c, K * N * c
        with torch.cuda.stream(cin):
            if i >= nslot:
                cin.wait_event(freed[i - nslot])
            dA[:na].copy_(hA[:na], non_blocking=True)
            h2d += 8 * na
            if kind == "tsmttsm" or beta != 0.0:
                dB[:nb].copy_(hB[:nb], non_blocking=True)
                h2d += 8 * nb
            if kind == "tsmm":
                dC[: M * N * c].copy_(hCin[: M * N * c], non_blocking=True)
                h2d += 8 * M * N * c
            copied[i].record(cin)
        compute.wait_event(copied[i])
        A = _mat(dA, K, M, cplx)
        if kind == "tsmttsm":
            out = torch.empty((M, N), dtype=A.dtype, device=dev)
            tsm.tsmttsm(A, _mat(dB, K, N, cplx), out, op="C" if cplx else "T")
            small_out.append(out)
            done[i].record(compute)
            freed[i] = done[i]
        else:
            tsm.tsmm(A, _mat(dC, M, N, cplx), _mat(dB, K, N, cplx), 1.0, beta)
            done[i].record(compute)
            with torch.cuda.stream(cout):
                cout.wait_event(done[i])
                hO[:nb].copy_(dB[:nb], non_blocking=True)
                d2h += 8 * nb
                freed[i].record(cout)
    hsmall = [torch.empty(o.shape, dtype=o.dtype, pin_memory=pinned) for o in small_out]
    for h, o in zip(hsmall, small_out):
        h.copy_(o, non_blocking=True)
        d2h += o.numel() * o.element_size()
    compute.wait_stream(cout)
    t1.record(compute)
    torch.cuda.synchronize()
    secs = t0.elapsed_time(t1) * 1e-3
    del slots, hA, hB, hO
    torch.cuda.empty_cache()
    return {"value": round(100.0 * ideal_s / secs, 3), "unit": "% of roofline", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": round(secs * 1e3, 1), "pinned": pinned}


# ------------------------------------------------------------------ extras

def _reps_for(t_ideal_s):
    """Timed calls per point: several for calls below a millisecond, so that
    the host's launch latency of the first one (the start event is recorded
    behind a single warm-up call, and that call cannot start before the
    event) is spread over them -- 32 below 100 us, 8 below 1 ms; one above."""
    if t_ideal_s > 1e-3:
        return 1
    return 8 if t_ideal_s > 1e-4 else 32


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


def _oracle_entries(cplx, M, N, K, dist, entries):
    """Entries (m, n) of op(A)^T B at full K computed by the oracle from the
    host generator's columns (never from the device), with the
    Cauchy-Schwarz scale ||a_m|| ||b_n|| of each."""
    import numpy as np
    import oracle
    import synth
    out = []
    for (m, n) in entries:
        a = synth.column(0, K, m, M, complex_=cplx, dist=dist)
        b = synth.column(1, K, n, N, complex_=cplx, dist=dist)
        out.append((oracle.dot("C" if cplx else "T", a, b), float(np.linalg.norm(a) * np.linalg.norm(b))))
    return out


def run_split_extra(flatA, flatB, K, bw):
    """Split-precision TSMTTSM on the split workload: time, speed-up over the
    plain FP64 path, HBM fraction, and the error of two sampled entries
    ((0, 0) and (M-1, N-1)) against the oracle's values at full K, relative
    to each entry and to its Cauchy-Schwarz scale ||a_m|| ||b_n||."""
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
            h1 = C1.cpu().numpy()
            ents = [(0, 0), (M - 1, N - 1)]
            ref = _oracle_entries(cplx, M, N, K, dist, ents)
            err_rel = max(abs(h1[m, n] - r) / abs(r) for (m, n), (r, _) in zip(ents, ref))
            err_cs = max(abs(h1[m, n] - r) / s for (m, n), (r, s) in zip(ents, ref))
            c = 2 if cplx else 1
            nbytes = 8.0 * c * (M + N) * K
            out.append({"dist": dist, "dtype": "c64" if cplx else "r64", "M": M, "N": N,
                        "ms_split": round(ms_s, 3), "ms_fp64": round(ms_d, 3), "speedup": round(ms_d / ms_s, 2),
                        "split_gbs": round(nbytes / (ms_s * 1e-3) / 1e9, 1),
                        "hbm_frac": round(nbytes / (ms_s * 1e-3) / 1e9 / bw, 3),
                        "oracle_entry_rel_err": err_rel, "oracle_entry_err_vs_norms": err_cs,
                        "rel_diff_vs_fp64_path": float(torch.linalg.norm(C1 - C2) / torch.linalg.norm(C2)),
                        "status": status})
    tsm.fill_random(flatA.view(K, 128), 0)
    tsm.fill_random(flatB.view(K, 128), 1)
    return out


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


GRID_STEP = 8


def run_grid_extra(flatA, flatB, K, bw, p64):
    """Non-square widths: TSMTTSM at every (M, N) with M, N multiples of 8 in
    8..64 (real op T and complex op C) at K = 2^24, percent of roofline per
    shape with the library's tuned choice; one warm-up and one timed call."""
    import torch
    import paper_1905_03136_gb300 as tsm
    res = {}
    below = []
    for cplx in (False, True):
        dt = torch.complex128 if cplx else torch.float64
        pct = []
        for M in range(GRID_STEP, 65, GRID_STEP):
            row = []
            for N in range(GRID_STEP, 65, GRID_STEP):
                A, B = _views(flatA, flatB, cplx, M, N, K)
                C = torch.zeros((M, N), dtype=dt, device=flatA.device)
                ms = _time(lambda: tsm.tsmttsm(A, B, C, op="C" if cplx else "T"), reps=1)
                p = 100.0 * ideal_seconds(cplx, M, N, K, bw, p64) / (ms * 1e-3)
                row.append(round(p, 1))
                if p < 90.0:
                    below.append("%s %dx%d: %.1f" % ("c64" if cplx else "r64", M, N, p))
            pct.append(row)
        flat = [x for r in pct for x in r]
        res["c64" if cplx else "r64"] = {"roofline_pct": pct, "median": statistics.median(flat), "min": min(flat)}
    res["what"] = "TSMTTSM % of roofline, rows M = 8, 16, ..., 64, columns N = 8, 16, ..., 64, K = 2^24"
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
    # small K: the step against its two products timed alone (the gap is
    # what a single fused kernel could remove at most: one launch and the C
    # round trip through L2)
    small = []
    for (cplx, M, N) in ((True, 32, 32), (False, 8, 8), (True, 64, 64)):
        c = 2 if cplx else 1
        for Ks in (3000, 10 ** 4, 1 << 15, 10 ** 5, 10 ** 6):
            A = flatA[: Ks * M * c]
            B = Bw[: Ks * N * c]
            B.copy_(flatB[: Ks * N * c])
            if cplx:
                A, B = A.view(torch.complex128), B.view(torch.complex128)
            A, B = A.view(Ks, M), B.view(Ks, N)
            C = torch.empty((M, N), dtype=A.dtype, device=A.device)
            t_gs = _time(lambda: tsm.gs_step(A, B, C), reps=50, warm=5)
            t_two = _time(lambda: tsm.gs_step(A, B, C, mode="two_products"), reps=50, warm=5)
            t_fused = _time(lambda: tsm.gs_step(A, B, C, mode="fused"), reps=50, warm=5)
            t_1 = _time(lambda: tsm.tsmttsm(A, B, C, op="C"), reps=50, warm=5)
            t_2 = _time(lambda: tsm.tsmm(A, C, B, -1.0, 1.0), reps=50, warm=5)
            small.append({"dtype": "c64" if cplx else "r64", "M": M, "N": N, "K": Ks, "gs_us": round(t_gs * 1e3, 2),
                          "two_products_us": round(t_two * 1e3, 2), "fused_us": round(t_fused * 1e3, 2),
                          "tsmttsm_us": round(t_1 * 1e3, 2), "tsmm_us": round(t_2 * 1e3, 2)})
    tsm.gs_status()
    del Bw
    torch.cuda.empty_cache()
    return {"what": "tsm_gs_step: TSMTTSM (op C) then TSMM (alpha=-1, beta=1) on one stream, C on the device; "
                    "small_k: the default path (fused for K <= 2^15), the two products, the fused kernel, and "
                    "each product alone",
            "roofline_pct_all": 100 * ideal / meas, "calls": out, "small_k": small}


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
             8: (5, 2, 2), 9: (3, 5, 1), 10: (5, 3, 1), 11: (2, 7, 1), 12: (7, 2, 1), 13: (8, 8, 1), 14: (5, 5, 1)}
    tprs = {1: 4, 2: 8, 3: 16}
    rt = {v["dtype"]: v["index"] for v in tsm.variants(tsm.KIND_TSMM) if v["name"].endswith("_rt_npt4_u2")}
    cfg = []
    for (kind, cplx, M, N, K) in insts:
        cands, feats = [], []
        if kind == 0:
            for code, (tm, tn, u) in tiles.items():
                if cplx and code in (4, 5, 13, 14):
                    continue  # complex runs these codes as codes 3 and 6
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


def batched_views(flatA, flatB, insts):
    """Device views (A, B, out) of every batched instance: A and B read the
    two seeded pools, every output has its own buffer."""
    import torch
    dev = flatA.device
    views = []
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
    return views


BATCHED_TILE_CODES = range(1, 15)
BATCHED_TPR_CODES = range(1, 5)


def batched_make(insts, views, cfgs):
    from paper_1905_03136_gb300 import batched as bt
    descs = [bt.desc(k, A, B, O, 1.0, 0.0, ("C" if c else "T") if k == 0 else "N", cfg)
             for (k, c, M, N, K), (A, B, O), cfg in zip(insts, views, cfgs)]
    return bt.Batch(descs)


def batched_configs_exhaustive(insts, flatA, flatB, k_probe=1 << 19):
    """Exhaustive per-instance configuration: for every distinct instance
    shape (kind, dtype, M, N), each configuration code of the batched kernel
    is timed on a one-shape batch of `k_probe` rows cut into 1024-row items
    (enough items for every persistent CTA, so the time is the code's
    throughput, not one item's latency); the fastest code is kept."""
    best = {}
    for inst in insts:
        key = tuple(inst[:4])
        if key in best:
            continue
        kind, cplx = key[0], key[1]
        probe = key + (k_probe,)
        v = batched_views(flatA, flatB, [probe])
        times = {}
        for code in (BATCHED_TILE_CODES if kind == 0 else BATCHED_TPR_CODES):
            if kind == 0 and code_tile_threads(code, cplx, key[2], key[3]) > 256:
                continue
            b = batched_make([probe], v, [code | (10 << 8)])
            times[code] = _time(b.run, reps=2)
            b.close()
        best[key] = min(times, key=times.get)
        del v
    return [best[tuple(i[:4])] for i in insts], len(best)


def code_tile_threads(code, cplx, M, N):
    """Threads per row lane of a batched TSMTTSM tile code (the kernel falls
    back to its default for a code above 256)."""
    tiles = {1: (1, 1), 2: (2, 2), 3: (4, 4), 4: (4, 8), 5: (8, 4), 6: (3, 3), 7: (2, 5), 8: (5, 2), 9: (3, 5),
             10: (5, 3), 11: (2, 7), 12: (7, 2), 13: (8, 8), 14: (5, 5)}
    tm, tn = tiles[code]
    if cplx and code in (4, 5, 13):
        tm = tn = 4
    if cplx and code == 14:
        tm = tn = 3
    return math.ceil(M / tm) * math.ceil(N / tn)


def run_batched_extra(flatA, flatB, exhaustive=True):
    """256 instances in one graph launch: the default configurations, the cost
    model's and the exhaustive per-instance best (every code timed per shape),
    against launching every instance separately with the library's own
    choices."""
    import torch
    from paper_1905_03136_gb300 import costmodel as cm
    import paper_1905_03136_gb300 as tsm
    insts = batched_workload()
    views = batched_views(flatA, flatB, insts)
    flops = sum(2.0 * M * N * K * (4 if c else 1) for (_, c, M, N, K) in insts)
    res = {"instances": len(insts), "flops": flops}

    default = batched_make(insts, views, [0] * len(insts))
    res["items"], res["ctas"] = default.info()
    res["default_graph_ms"] = _time(default.run, reps=2)
    res["default_direct_ms"] = _time(default.run_direct, reps=1)
    default.close()
    model_path = os.path.join(ROOT, "paper_1905_03136_gb300", "tuning", "costmodel.npz")
    mlp_cfg = None
    if os.path.exists(model_path):
        model = cm.CostModel()
        model.load(model_path)
        mlp_cfg = batched_configs_from_model(insts, model)
        b = batched_make(insts, views, mlp_cfg)
        res["mlp_graph_ms"] = _time(b.run, reps=2)
        b.close()
    if exhaustive:
        t0 = time.time()
        ex_cfg, shapes = batched_configs_exhaustive(insts, flatA, flatB)
        res["exhaustive_search_s"] = round(time.time() - t0, 1)
        res["exhaustive_shapes"] = shapes
        b = batched_make(insts, views, ex_cfg)
        res["exhaustive_graph_ms"] = _time(b.run, reps=2)
        b.close()
        if mlp_cfg is not None:
            res["mlp_same_code_as_exhaustive"] = sum(a == e for a, e in zip(mlp_cfg, ex_cfg))
            res["mlp_over_exhaustive"] = res["mlp_graph_ms"] / res["exhaustive_graph_ms"]

    def separate():
        for (k, c, M, N, K), (A, B, O) in zip(insts, views):
            if k == 0:
                tsm.tsmttsm(A, B, O, op="C" if c else "T")
            else:
                tsm.tsmm(A, B, O)
    res["separate_launches_ms"] = _time(separate, reps=1)
    res["gflops_default_graph"] = flops / (res["default_graph_ms"] * 1e-3) / 1e9
    del views
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


def run_extras(args, flatA, flatB, K, bw, p64, emit):
    """Runs every extra, emits each one, and returns the short summary the
    headline line carries."""
    summ = {}

    def guarded(name, fn):
        try:
            rec = fn()
        except Exception as e:  # reported, never hidden
            rec = {"error": repr(e)}
        emit(name, rec if isinstance(rec, dict) else {"rows": rec})
        return rec

    w = guarded("widths", lambda: run_widths_extra(flatA, flatB, K, bw, p64))
    if "error" not in w:
        summ["widths"] = {kind: {dt: [statistics.median(w[kind][dt]["roofline_pct"]), w[kind][dt]["min_pct"],
                                      [i + 1 for i, p in enumerate(w[kind][dt]["roofline_pct"]) if p < 90.0]]
                                 for dt in ("r64", "c64")} for kind in ("tsmttsm", "tsmm_beta0", "tsmm_beta1")}
        summ["widths"]["what"] = "M=N=w, w=1..64: [median %, min %, widths below 90 %]"
    g = guarded("grid", lambda: run_grid_extra(flatA, flatB, K, bw, p64))
    if "error" not in g:
        summ["grid_8"] = {dt: [g[dt]["median"], g[dt]["min"]] for dt in ("r64", "c64")}
        summ["grid_8"]["below_90"] = len(g["below_90"])
    sp = guarded("split", lambda: run_split_extra(flatA, flatB, K, bw))
    if isinstance(sp, list):
        summ["split"] = {"%s %dx%d %s" % (r["dtype"], r["M"], r["N"], r["dist"][:4]):
                         [r["ms_split"], r["speedup"], float("%.2g" % r["oracle_entry_err_vs_norms"])]
                         for r in sp}
        summ["split"]["what"] = "[ms, speed-up over FP64, max sampled-entry error vs oracle / (|a_m||b_n|)]"
    cb = guarded("cublas", lambda: run_cublas_extra(flatA, flatB, K, bw, p64))
    if "value" in cb:
        summ["cublas_tsmttsm_pct"] = round(cb["value"], 2)
    gs = guarded("gs_step", lambda: run_gs_extra(flatA, flatB, K, bw, p64))
    if "roofline_pct_all" in gs:
        summ["gs_step_pct"] = round(gs["roofline_pct_all"], 2)
    guarded("small_k_ramp", lambda: run_ramp_extra(flatA, flatB, bw, p64))
    bt = guarded("batched", lambda: run_batched_extra(flatA, flatB))
    if "separate_launches_ms" in bt:
        summ["batched_ms"] = {k[:-3]: round(bt[k], 1) for k in ("default_graph_ms", "mlp_graph_ms",
                                                                 "exhaustive_graph_ms", "separate_launches_ms")
                              if k in bt}
    return summ


def main():
    ap = argparse.ArgumentParser(description="TSMTTSM / TSMM roofline sweep benchmark")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--cpu-rows", type=int, default=1 << 17, help="rows per call of the 1-thread CPU sample")
    ap.add_argument("--cpu-rows-all", type=int, default=1 << 19, help="rows per call of the all-cores CPU sample")
    ap.add_argument("--ref-rows", type=int, default=1 << 17, help="rows per call per reference-arm step")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the per-width / split / batched extras")
    ap.add_argument("--extras-out", default=None, help="also write every extra to this JSON file")
    ap.add_argument("--case", default=None, help="profile one config, e.g. c64:64x64")
    ap.add_argument("--k", type=int, default=1 << 20, help="rows for --case")
    ap.add_argument("--split", action="store_true", help="--case: use the split-precision path")
    ap.add_argument("--tsmm", action="store_true", help="--case: TSMM instead of TSMTTSM")
    ap.add_argument("--beta", type=float, default=0.0, help="--case --tsmm: beta")
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
