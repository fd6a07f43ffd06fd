"""The cost model's network kernels against the float64 oracle: forward
values, gradient of the mean squared error, one Adam step, reproducible
training; and the learned tuner's regret against exhaustive search."""

import os

import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import paper_1905_03136_gb300 as t
    from paper_1905_03136_gb300 import build, _lib, mlp
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    t.load()
    return mlp


def _case(D=17, H=64, n=300, seed=3):
    rng = np.random.default_rng(seed)
    p = rng.uniform(-0.3, 0.3, omlp.param_count(D, H)).astype(np.float32)
    X = rng.uniform(-1, 1, (n, D)).astype(np.float32)
    t = rng.uniform(-1, 1, n).astype(np.float32)
    return p, X, t


def test_forward_and_gradient_match_oracle(M):
    import torch
    D, H = 17, 64
    p, X, t = _case(D, H)
    net = M.Mlp(D, H, max_batch=1024)
    net.set_params(p)
    dX, dt = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    y = net.forward(dX).cpu().numpy()
    y_ref = omlp.forward(p, X, D, H)
    assert np.max(np.abs(y - y_ref)) <= 1e-5 * max(1.0, np.max(np.abs(y_ref)))
    loss = float(net.backward(dX, dt).item())
    assert abs(loss - omlp.loss(p, X, t, D, H)) <= 1e-5 * max(1.0, loss)
    g = net.grads().astype(np.float64)
    g_ref = omlp.grad(p, X, t, D, H)
    assert np.max(np.abs(g - g_ref)) <= 1e-4 * np.max(np.abs(g_ref))
    # the oracle's gradient itself against central differences in float64
    i = int(np.argmax(np.abs(g_ref)))
    e = np.zeros_like(g_ref)
    e[i] = 1e-6
    fd = (omlp.loss(p.astype(np.float64) + e, X, t, D, H) - omlp.loss(p.astype(np.float64) - e, X, t, D, H)) / 2e-6
    assert abs(fd - g_ref[i]) <= 1e-6 * abs(g_ref[i]) + 1e-12


def test_adam_step_matches_oracle(M):
    import torch
    D, H = 5, 8
    p, X, t = _case(D, H, n=50)
    net = M.Mlp(D, H, max_batch=64)
    net.set_params(p)
    net.backward(torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda())
    g = net.grads().astype(np.float64)
    net.adam(lr=1e-2)
    torch.cuda.synchronize()
    p_ref, _, _ = omlp.adam(p.astype(np.float64), g, 0.0, 0.0, 1, 1e-2)
    assert np.max(np.abs(net.params() - p_ref)) <= 1e-6


def test_training_is_reproducible_and_learns(M):
    import torch
    rng = np.random.default_rng(5)
    X = rng.uniform(-1, 1, (2000, 6)).astype(np.float32)
    t = (np.sin(2 * X[:, 0]) + X[:, 1] * X[:, 2]).astype(np.float32)
    dX, dt = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    a = M.Mlp(6, 64, max_batch=4096, seed=11)
    b = M.Mlp(6, 64, max_batch=4096, seed=11)
    ha = a.fit(dX, dt, epochs=600, lr=3e-3)
    hb = b.fit(dX, dt, epochs=600, lr=3e-3)
    assert np.array_equal(a.params(), b.params())
    assert ha[-1] < 0.1 * ha[0]


def test_learned_tuner_regret_on_held_out_shapes(M):
    """Trained (by the GPU kernels) on the autotuner's timing log minus
    held-out shapes.  (1) For each held-out shape the logged time of the
    model's pick over the logged exhaustive best must stay within 5%
    (geometric mean).  (2) What the model gains over the library's built-in
    heuristic (its choice without a tuning table): both picks are timed now,
    on this GPU, for every held-out shape, and the model's picks must take
    less time in total and in geometric mean."""
    import torch
    import paper_1905_03136_gb300 as tsm
    from paper_1905_03136_gb300 import costmodel as cm
    log = os.path.join(os.path.dirname(cm.__file__), "tuning", "timing_log.jsonl")
    if not os.path.exists(log):
        pytest.skip("no timing log committed yet")
    recs = cm.load_log(log)
    shapes = sorted({cm.shape_key(r) for r in recs})
    held = [s for i, s in enumerate(shapes) if i % 5 == 2]
    train = [r for r in recs if cm.shape_key(r) not in set(held)]
    model = cm.CostModel(seed=1)
    model.fit(train, epochs=3000)
    ev = cm.evaluate(model, recs, held)
    mlp_geo = ev["mlp_regret_geomean"]
    assert mlp_geo <= 1.05, (mlp_geo, sorted(r["mlp_regret"] for r in ev["rows"])[-5:])

    Kmax = max(s[4] for s in held)
    flatA = torch.empty(Kmax * 128, dtype=torch.float64, device="cuda")
    flatB = torch.empty(Kmax * 128, dtype=torch.float64, device="cuda")
    tsm.fill_random(flatA.view(Kmax, 128), 0)
    tsm.fill_random(flatB.view(Kmax, 128), 1)
    index = {k: {v["name"]: v["index"] for v in tsm.variants(k)} for k in (tsm.KIND_TSMTTSM, tsm.KIND_TSMM)}
    by_shape = {}
    for r in recs:
        by_shape.setdefault(cm.shape_key(r), []).append(r)
    t_mlp, t_heur, ratios = 0.0, 0.0, []
    for key in held:
        kind, cplx, Mm, Nn, K = key
        rs = by_shape[key]
        pick = rs[int(np.argmin(model.predict_log2_ineff([cm.record_features(r) for r in rs])))]
        hname, hgrid = cm.heuristic_pick(kind, cplx, Mm, Nn, K)
        c = 2 if cplx else 1
        dt = torch.complex128 if cplx else torch.float64
        X = flatA[: K * Mm * c].view(dt).view(K, Mm) if cplx else flatA[: K * Mm].view(K, Mm)
        if kind == 0:
            Y = flatB[: K * Nn * c]
            Z = torch.zeros((Mm, Nn), dtype=dt, device="cuda")
            Y = (Y.view(dt) if cplx else Y).view(K, Nn)
        else:
            Y = flatB[: Mm * Nn * c].clone()
            Y = (Y.view(dt) if cplx else Y).view(Mm, Nn)
            Z = torch.empty((K, Nn), dtype=dt, device="cuda")
        vk = tsm.KIND_TSMTTSM if kind == 0 else tsm.KIND_TSMM
        ms = [tsm.time_variant(kind, X, Y, Z, index[vk][name], grid, reps=2)
              for name, grid in ((pick["variant"], pick["grid"]), (hname, hgrid))]
        t_mlp += ms[0]
        t_heur += ms[1]
        ratios.append(ms[0] / ms[1])
        del X, Y, Z
    geo = float(np.exp(np.mean(np.log(ratios))))
    print("held-out shapes %d: logged regret geomean MLP %.4f (max %.3f); timed now: MLP %.2f ms, heuristic "
          "%.2f ms, geomean MLP/heuristic %.4f" % (len(held), mlp_geo, ev["mlp_regret_max"], t_mlp, t_heur, geo))
    assert t_mlp < t_heur and geo < 1.0, (t_mlp, t_heur, geo)
