"""Exhaustive autotuning driver (Sec. 5.1 and 7 of the paper).

For each requested shape this fills device buffers with the seeded synthetic
inputs, runs the library's exhaustive search (``tsm_tune``: every variant
that supports the shape at several grid sizes, timed with CUDA events),
keeps the winner in the tuning table and appends every measurement to a
timing log.  The log (one JSON object per line) is the training set of the
learned cost model (``mlp.py``); the table is what the library consults
before its built-in heuristic.

Usage:
  python -m paper_1905_03136_gb300.autotune --K 16777216 --table T.txt --log L.jsonl [--kind tsmttsm|tsmm|both]
         [--shapes r64:1x1,c64:2x2] [--keep-table]
"""

import argparse
import json
import os
import sys
import time

SQUARE = (1, 2, 4, 8, 16, 32, 64)
TSMTTSM_OFFDIAG = ((1, 64), (64, 1), (8, 32), (32, 8))
TSMM_OFFDIAG = ((4, 64), (64, 4))

PKG = os.path.dirname(os.path.abspath(__file__))
DEFAULT_TABLE = os.path.join(PKG, "tuning", "gb300_sm103.txt")


def sweep_shapes(kind):
    off = TSMTTSM_OFFDIAG if kind == 0 else TSMM_OFFDIAG
    return [(c, m, n) for c in (False, True) for (m, n) in [(w, w) for w in SQUARE] + list(off)]


def tune_shapes(kind, shapes, K, reps=3, log=None, flat=None):
    """Runs tsm_tune for each (cplx, M, N) and returns the log records."""
    import torch
    import paper_1905_03136_gb300 as tsm
    tsm.load()
    info = {v["index"]: v for v in tsm.variants(kind)}
    if flat is None:
        flatA = torch.empty(K * 128, dtype=torch.float64, device="cuda")
        flatB = torch.empty(K * 128, dtype=torch.float64, device="cuda")
        tsm.fill_random(flatA.view(K, 128), 0)
        tsm.fill_random(flatB.view(K, 128), 1)
    else:
        flatA, flatB = flat
    records = []
    for (cplx, M, N) in shapes:
        c = 2 if cplx else 1
        X = flatA[: K * M * c]
        if kind == 0:
            Y = flatB[: K * N * c]
            Z = torch.zeros(M * N * c, dtype=torch.float64, device="cuda")
        else:
            Y = flatB[: M * N * c]
            Z = torch.empty(K * N * c, dtype=torch.float64, device="cuda")
        if cplx:
            X, Y, Z = (t.view(torch.complex128) for t in (X, Y, Z))
        X = X.view(K, M)
        Y = Y.view(K, N) if kind == 0 else Y.view(M, N)
        Z = Z.view(M, N) if kind == 0 else Z.view(K, N)
        t0 = time.time()
        samples = tsm.tune(kind, X, Y, Z, reps=reps)
        for (v, g, ms) in samples:
            vi = info[v] if not info[v].get("runtime_tile") else tsm.variant_shape(kind, v, int(cplx), M, N)
            rec = {"kind": kind, "dtype": int(cplx), "M": M, "N": N, "K": K, "variant": vi["name"],
                   "tile_m": vi["tile_m"], "tile_n": vi["tile_n"], "tpr": vi["threads_per_row"],
                   "unroll": vi["unroll"], "generated": vi["generated"], "fixed": int(vi["fixed_m"] > 0),
                   "grid": g, "ms": ms}
            records.append(rec)
            if log is not None:
                log.write(json.dumps(rec) + "\n")
        if log is not None:
            log.flush()
        best = min(samples, key=lambda s: s[2])
        print("%s %s %dx%d best %s grid=%d %.4f ms (%d samples, %.1fs)" % (
            "tsmttsm" if kind == 0 else "tsmm", "c64" if cplx else "r64", M, N, info[best[0]]["name"],
            best[1], best[2], len(samples), time.time() - t0), flush=True)
        del X, Y, Z
    return records


def main():
    ap = argparse.ArgumentParser(description="exhaustive autotuning of libtsm variants")
    ap.add_argument("--K", type=int, default=1 << 24)
    ap.add_argument("--kind", choices=("tsmttsm", "tsmm", "both"), default="both")
    ap.add_argument("--table", default=DEFAULT_TABLE)
    ap.add_argument("--log", default=None, help="append measurements (JSON lines) here")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--random", type=int, default=0,
                    help="tune this many random (dtype, M, N) shapes instead of the sweep")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--shapes", default=None,
                    help="comma-separated shapes to tune instead of the sweep, e.g. r64:1x1,c64:2x2")
    ap.add_argument("--keep-table", action="store_true", help="merge into the loaded table")
    args = ap.parse_args()
    import torch
    import paper_1905_03136_gb300 as tsm
    lib = tsm.load()
    if not args.keep_table:
        lib.tsm_clear_tuning()
    log = open(args.log, "a") if args.log else None
    K = args.K
    flatA = torch.empty(K * 128, dtype=torch.float64, device="cuda")
    flatB = torch.empty(K * 128, dtype=torch.float64, device="cuda")
    tsm.fill_random(flatA.view(K, 128), 0)
    tsm.fill_random(flatB.view(K, 128), 1)
    kinds = {"tsmttsm": [0], "tsmm": [1], "both": [0, 1]}[args.kind]
    import numpy as np
    rng = np.random.default_rng(args.seed)
    for kind in kinds:
        if args.shapes:
            shapes = []
            for item in args.shapes.split(","):
                dt, wh = item.split(":")
                m, n = (int(x) for x in wh.split("x"))
                shapes.append((dt == "c64", m, n))
        elif args.random:
            shapes = [(bool(rng.integers(0, 2)), int(rng.integers(1, 65)), int(rng.integers(1, 65)))
                      for _ in range(args.random)]
        else:
            shapes = sweep_shapes(kind)
        tune_shapes(kind, shapes, K, args.reps, log, (flatA, flatB))
    os.makedirs(os.path.dirname(os.path.abspath(args.table)), exist_ok=True)
    tsm._lib.call("tsm_save_tuning", args.table.encode())
    print("table written to", args.table)


if __name__ == "__main__":
    sys.path.insert(0, os.path.dirname(PKG))
    main()
