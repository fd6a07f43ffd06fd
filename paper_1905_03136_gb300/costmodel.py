"""Learned cost model for kernel-configuration choice.

The paper picks each size's configuration by exhaustive search and proposes
a performance model to prune candidates faster (Sec. 7).  Here a small MLP
(``mlp.Mlp``: 3 layers, 64 hidden, FP32, trained by the library's own CUDA
kernels) learns, from the autotuner's timing log, the function

    (product, dtype, M, N, K, variant attributes, grid) -> log2(time / roofline time)

i.e. how far a configuration stays from the roofline bound of Eq. 1.  For an
unseen shape it scores every candidate the exhaustive search would time
(every supporting variant at the tuner's grid sizes) and keeps the argmin;
exhaustive tuning remains the fallback and the yardstick of its regret.
"""

import json
import math

import numpy as np

HBM_GBS = 6790.0
FP64_GFLOPS = 1250.0
SM_COUNT = 152


def roofline_ms(kind, cplx, M, N, K, hbm_gbs=HBM_GBS, fp64_gflops=FP64_GFLOPS):
    """Lower bound of Eq. 1: max(bytes / bandwidth, flops / FP64 peak)."""
    c = 2 if cplx else 1
    flops = 2.0 * M * N * K * (4 if cplx else 1)
    nbytes = 8.0 * c * (M * K + N * K + M * N)
    return 1e3 * max(nbytes / (hbm_gbs * 1e9), flops / (fp64_gflops * 1e9))


def featurize(kind, cplx, M, N, K, tile_m, tile_n, tpr, unroll, generated, fixed, grid, sm=SM_COUNT):
    c = 2 if cplx else 1
    flops = 2.0 * M * N * K * (4 if cplx else 1)
    nbytes = 8.0 * c * (M * K + N * K + M * N)
    f = [float(kind), float(cplx), math.log2(M) / 6, math.log2(N) / 6, (math.log2(K) - 20) / 4,
         math.log2(grid / sm) / 3, math.log2(flops / nbytes) / 4]
    if kind == 0:
        pm, pn = math.ceil(M / tile_m), math.ceil(N / tile_n)
        P = pm * pn
        lanes = max(256 // P, 1)
        waste = pm * tile_m * pn * tile_n / (M * N)
        f += [tile_m / 8, tile_n / 8, 0.0, 0.0, math.log2(P) / 8, math.log2(lanes) / 8, waste - 1]
    else:
        npt = math.ceil(N / tpr)
        waste = npt * tpr / N
        f += [0.0, 0.0, math.log2(tpr) / 5, npt / 16, 0.0, math.log2(256 // tpr) / 8, waste - 1]
    f += [unroll / 4, float(generated), float(fixed)]
    return np.array(f, dtype=np.float32)


N_FEATURES = 17


def record_features(r):
    return featurize(r["kind"], r["dtype"], r["M"], r["N"], r["K"], max(r["tile_m"], 1), max(r["tile_n"], 1),
                     max(r["tpr"], 1), r["unroll"], r["generated"], r["fixed"], r["grid"])


def record_target(r):
    return math.log2(r["ms"] / roofline_ms(r["kind"], r["dtype"], r["M"], r["N"], r["K"]))


def load_log(paths):
    recs = []
    for p in paths if isinstance(paths, (list, tuple)) else [paths]:
        with open(p) as f:
            for line in f:
                line = line.strip()
                if line:
                    recs.append(json.loads(line))
    return recs


def shape_key(r):
    return (r["kind"], r["dtype"], r["M"], r["N"], r["K"])


class CostModel:
    """MLP on standardized targets; trained and evaluated on the GPU."""

    def __init__(self, hidden=64, seed=0):
        from .mlp import Mlp
        self.net = Mlp(N_FEATURES, hidden, max_batch=1 << 16, seed=seed)
        self.mu, self.sigma = 0.0, 1.0

    def fit(self, records, epochs=3000, lr=3e-3):
        import torch
        X = torch.from_numpy(np.stack([record_features(r) for r in records])).cuda()
        y = np.array([record_target(r) for r in records], dtype=np.float32)
        self.mu, self.sigma = float(y.mean()), float(y.std() + 1e-6)
        t = torch.from_numpy((y - self.mu) / self.sigma).cuda()
        return self.net.fit(X, t, epochs=epochs, lr=lr)

    def predict_log2_ineff(self, feats):
        import torch
        X = torch.from_numpy(np.ascontiguousarray(np.stack(feats))).cuda()
        y = self.net.forward(X).cpu().numpy().astype(np.float64)
        return y * self.sigma + self.mu

    def predict_ms(self, kind, cplx, M, N, K, feats):
        return roofline_ms(kind, cplx, M, N, K) * np.exp2(self.predict_log2_ineff(feats))

    def save(self, path):
        np.savez(path, params=self.net.params(), mu=self.mu, sigma=self.sigma)

    def load(self, path):
        d = np.load(path)
        self.net.set_params(d["params"])
        self.mu, self.sigma = float(d["mu"]), float(d["sigma"])


def candidates(kind, cplx, M, N):
    """(variant, grid) pairs the exhaustive tuner would time; each variant is
    described for this shape (runtime-tile variants with the tile their
    launch picks)."""
    import ctypes
    import paper_1905_03136_gb300 as tsm
    from . import _lib
    lib = tsm.load()
    out = []
    for v in tsm.variants(kind):
        if not lib.tsm_variant_supports(kind, v["index"], int(cplx), M, N):
            continue
        v = tsm.variant_shape(kind, v["index"], int(cplx), M, N)
        grids = (ctypes.c_int * 4)()
        n = ctypes.c_int()
        _lib.call("tsm_tune_grids", kind, v["index"], int(cplx), M, N, grids, 4, ctypes.byref(n))
        for g in grids[: n.value]:
            out.append((v, g))
    return out


def choose(model, kind, cplx, M, N, K):
    """The MLP's pick: (variant dict, grid, predicted ms)."""
    cands = candidates(kind, cplx, M, N)
    feats = [featurize(kind, int(cplx), M, N, K, max(v["tile_m"], 1), max(v["tile_n"], 1),
                       max(v["threads_per_row"], 1), v["unroll"], v["generated"], int(v["fixed_m"] > 0), g)
             for v, g in cands]
    ms = model.predict_ms(kind, int(cplx), M, N, K, feats)
    i = int(np.argmin(ms))
    return cands[i][0], cands[i][1], float(ms[i])


def regret_from_log(model, records, shapes):
    """For each shape (key) of `shapes`: the logged time of the MLP's choice
    over the logged exhaustive best.  Uses only the log (no new timing)."""
    by_shape = {}
    for r in records:
        by_shape.setdefault(shape_key(r), []).append(r)
    out = {}
    for key in shapes:
        rs = by_shape[key]
        feats = [record_features(r) for r in rs]
        pred = model.predict_log2_ineff(feats)
        pick = rs[int(np.argmin(pred))]
        best = min(r["ms"] for r in rs)
        out[key] = pick["ms"] / best
    return out


def heuristic_pick(kind, cplx, M, N, K):
    """(variant name, grid) the library picks WITHOUT a tuning table or model
    (its built-in rule); the table is restored afterwards."""
    import os
    import tempfile
    import paper_1905_03136_gb300 as tsm
    from . import _lib
    lib = tsm.load()
    fd, path = tempfile.mkstemp(suffix=".txt")
    os.close(fd)
    try:
        _lib.call("tsm_save_tuning", path.encode())
        lib.tsm_clear_tuning()
        v, g = tsm.choose(kind, int(cplx), M, N, K)
        name = tsm.variants(kind)[v]["name"]
        _lib.call("tsm_load_tuning", path.encode())
    finally:
        os.unlink(path)
    return name, g


def evaluate(model, records, held):
    """Held-out shapes: logged time of the model's pick, of the heuristic's
    pick and of the exhaustive best.  Returns a summary dict."""
    by_shape = {}
    for r in records:
        by_shape.setdefault(shape_key(r), []).append(r)
    rows = []
    for key in held:
        rs = by_shape[key]
        pred = model.predict_log2_ineff([record_features(r) for r in rs])
        pick = rs[int(np.argmin(pred))]
        best = min(r["ms"] for r in rs)
        kind, cplx, M, N, K = key
        hname, hgrid = heuristic_pick(kind, cplx, M, N, K)
        hrec = [r for r in rs if r["variant"] == hname and r["grid"] == hgrid]
        hms = hrec[0]["ms"] if hrec else float("nan")
        rows.append({"shape": list(key), "best_ms": best, "mlp_ms": pick["ms"], "heuristic_ms": hms,
                     "mlp_regret": pick["ms"] / best, "heuristic_regret": hms / best})
    mr = np.array([r["mlp_regret"] for r in rows])
    hr = np.array([r["heuristic_regret"] for r in rows])
    ok = ~np.isnan(hr)
    return {"held_out_shapes": len(rows), "mlp_regret_geomean": float(np.exp(np.mean(np.log(mr)))),
            "mlp_regret_max": float(mr.max()),
            "heuristic_regret_geomean": float(np.exp(np.mean(np.log(hr[ok])))) if ok.any() else None,
            "mlp_total_ms": float(sum(r["mlp_ms"] for r in rows)),
            "heuristic_total_ms": float(np.nansum([r["heuristic_ms"] for r in rows])),
            "best_total_ms": float(sum(r["best_ms"] for r in rows)), "rows": rows}


def main():
    import argparse
    import os
    import sys
    ap = argparse.ArgumentParser(description="train the cost model on autotuner timing logs")
    ap.add_argument("logs", nargs="+")
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning",
                                                  "costmodel.npz"))
    ap.add_argument("--epochs", type=int, default=3000)
    ap.add_argument("--holdout", type=int, default=5, help="every n-th shape is held out (0: none)")
    args = ap.parse_args()
    recs = load_log(args.logs)
    shapes = sorted({shape_key(r) for r in recs})
    held = [s for i, s in enumerate(shapes) if args.holdout and i % args.holdout == 2]
    train = [r for r in recs if shape_key(r) not in set(held)]
    model = CostModel(seed=1)
    hist = model.fit(train, epochs=args.epochs)
    print("records %d shapes %d train %d held %d loss %.4f -> %.4f" % (len(recs), len(shapes), len(train),
                                                                      len(held), hist[0], hist[-1]))
    if held:
        ev = evaluate(model, recs, held)
        print(json.dumps({k: v for k, v in ev.items() if k != "rows"}))
    # the shipped model is trained on every shape
    full = CostModel(seed=1)
    full.fit(recs, epochs=args.epochs)
    full.save(args.out)
    print("saved", args.out)
    sys.stdout.flush()


if __name__ == "__main__":
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    main()
