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
         [--shapes r64:1x1,c64:2x2 | --widths 1-64] [--keep-table] [--skip-tuned] [--pruned TOPK]
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


def _operands(kind, cplx, M, N, K, flatA, flatB):
    """Views of the seeded flat buffers as the X, Y, Z arguments of tsm_tune
    (TSMTTSM: A, B, C; TSMM: A, C, B)."""
    import torch
    c = 2 if cplx else 1
    X = flatA[: K * M * c]
    if kind == 0:
        Y = flatB[: K * N * c]
        Z = torch.zeros(M * N * c, dtype=torch.float64, device=flatA.device)
    else:
        Y = flatB[: M * N * c]
        # kind 2 (TSMM with beta = 1) reads B: finite values
        Z = (torch.zeros if kind == 2 else torch.empty)(K * N * c, dtype=torch.float64, device=flatA.device)
    if cplx:
        X, Y, Z = (t.view(torch.complex128) for t in (X, Y, Z))
    X = X.view(K, M)
    Y = Y.view(K, N) if kind == 0 else Y.view(M, N)
    Z = Z.view(M, N) if kind == 0 else Z.view(K, N)
    return X, Y, Z


def tune_pruned(kind, shapes, K, model, topk=5, reps=1, log=None, flat=None, with_fixed=False):
    """Model-pruned search (the performance-model use the paper's Sec. 7
    proposes): the cost model ranks every (variant, grid) candidate the
    exhaustive search would time, only the `topk` best-ranked are timed, and
    the fastest of those enters the tuning table with its measured time.
    With `with_fixed`, the kernels specialised to the shape (generated or
    narrow) are timed as well, whatever their rank."""
    import numpy as np
    import paper_1905_03136_gb300 as tsm
    from . import _lib, costmodel
    tsm.load()
    flatA, flatB = flat
    records = []
    for (cplx, M, N) in shapes:
        t0 = time.time()
        cands = costmodel.candidates(kind, cplx, M, N)
        feats = [costmodel.featurize(kind, int(cplx), M, N, K, max(v["tile_m"], 1), max(v["tile_n"], 1),
                                     max(v["threads_per_row"], 1), v["unroll"], v["generated"],
                                     int(v["fixed_m"] > 0), g) for v, g in cands]
        pred = model.predict_ms(kind, int(cplx), M, N, K, feats)
        X, Y, Z = _operands(kind, cplx, M, N, K, flatA, flatB)
        timed = []
        pick = list(np.argsort(pred)[:topk])
        if with_fixed:
            # the kernels specialised to exactly this shape are always timed
            pick += [i for i, (v, g) in enumerate(cands) if v["fixed_m"] == M and v["fixed_n"] == N
                     and i not in pick]
        for i in pick:
            v, g = cands[int(i)]
            ms = tsm.time_variant(kind, X, Y, Z, v["index"], g, reps=reps)
            timed.append((ms, v, g, float(pred[int(i)])))
            rec = {"kind": kind, "dtype": int(cplx), "M": M, "N": N, "K": K, "variant": v["name"],
                   "tile_m": v["tile_m"], "tile_n": v["tile_n"], "tpr": v["threads_per_row"],
                   "unroll": v["unroll"], "generated": v["generated"], "fixed": int(v["fixed_m"] > 0),
                   "grid": g, "ms": ms}
            records.append(rec)
            if log is not None:
                log.write(json.dumps(rec) + "\n")
        if log is not None:
            log.flush()
        ms, v, g, p = min(timed, key=lambda x: x[0])
        _lib.call("tsm_set_tuning_timed", kind, int(cplx), M, N, K, v["index"], g, ms)
        print("%s %s %dx%d pruned best %s grid=%d %.4f ms (model %.4f; %d of %d timed, %.1fs)" % (
            ("tsmttsm", "tsmm", "tsmm_beta")[kind], "c64" if cplx else "r64", M, N, v["name"], g, ms, p,
            len(timed), len(cands), time.time() - t0), flush=True)
        del X, Y, Z
    return records


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
        X, Y, Z = _operands(kind, cplx, M, N, K, flatA, flatB)
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
            ("tsmttsm", "tsmm", "tsmm_beta")[kind], "c64" if cplx else "r64", M, N, info[best[0]]["name"],
            best[1], best[2], len(samples), time.time() - t0), flush=True)
        del X, Y, Z
    return records


def _has_entry(kind, shape, K):
    """True if the loaded tuning table has an entry for (kind, shape) in K's bucket."""
    import tempfile
    from . import _lib
    fd, path = tempfile.mkstemp(suffix=".txt")
    os.close(fd)
    try:
        _lib.call("tsm_save_tuning", path.encode())
        kb = K.bit_length() - 1
        cplx, M, N = shape
        with open(path) as f:
            for line in f:
                p = line.split()
                if len(p) == 8 and not line.startswith("#") and \
                        (int(p[0]), int(p[1]), int(p[2]), int(p[3]), int(p[4])) == (kind, int(cplx), M, N, kb):
                    return True
    finally:
        os.unlink(path)
    return False


def main():
    ap = argparse.ArgumentParser(description="exhaustive autotuning of libtsm variants")
    ap.add_argument("--K", type=int, default=1 << 24)
    ap.add_argument("--kind", choices=("tsmttsm", "tsmm", "tsmm_beta", "both"), default="both",
                    help="tsmm_beta: TSMM timed with beta = 1, kept under its own table key")
    ap.add_argument("--table", default=DEFAULT_TABLE)
    ap.add_argument("--log", default=None, help="append measurements (JSON lines) here")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--random", type=int, default=0,
                    help="tune this many random (dtype, M, N) shapes instead of the sweep")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--shapes", default=None,
                    help="comma-separated shapes to tune instead of the sweep, e.g. r64:1x1,c64:2x2")
    ap.add_argument("--keep-table", action="store_true", help="merge into the loaded table")
    ap.add_argument("--widths", default=None,
                    help="square shapes M = N = w for w in this range (e.g. 1-64), both dtypes")
    ap.add_argument("--skip-tuned", action="store_true",
                    help="leave shapes that already have an entry for this K bucket")
    ap.add_argument("--pruned", type=int, default=0,
                    help="time only the cost model's TOPK candidates per shape (0: exhaustive)")
    ap.add_argument("--model", default=os.path.join(PKG, "tuning", "costmodel.npz"))
    ap.add_argument("--with-fixed", action="store_true",
                    help="--pruned: also time every kernel specialised to the shape")
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
    kinds = {"tsmttsm": [0], "tsmm": [1], "tsmm_beta": [2], "both": [0, 1]}[args.kind]
    import numpy as np
    rng = np.random.default_rng(args.seed)
    for kind in kinds:
        if args.widths:
            lo, hi = (int(x) for x in args.widths.split("-"))
            shapes = [(c, w, w) for c in (False, True) for w in range(lo, hi + 1)]
        elif args.shapes:
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
        if args.skip_tuned:
            shapes = [sh for sh in shapes if not _has_entry(kind, sh, K)]
        if args.pruned:
            from .costmodel import CostModel
            model = CostModel()
            model.load(args.model)
            tune_pruned(kind, shapes, K, model, args.pruned, args.reps, log, (flatA, flatB), args.with_fixed)
        else:
            tune_shapes(kind, shapes, K, args.reps, log, (flatA, flatB))
    os.makedirs(os.path.dirname(os.path.abspath(args.table)), exist_ok=True)
    tsm._lib.call("tsm_save_tuning", args.table.encode())
    print("table written to", args.table)


if __name__ == "__main__":
    sys.path.insert(0, os.path.dirname(PKG))
    main()
